"""The allocation-free entry point, ofv_compute_noalloc.

It exists for callers that cannot call cudaMalloc: host programs whose device
memory belongs to another allocator (a framework's caching allocator, or a
pool sized at start-up), and real-time acquisition loops that forbid
allocation once running.  Its workspace is a fixed device array inside the
library instead of a handle's allocation.  These tests call it through the C
ABI and compare it with the handle-based ofv_compute on consecutive calls,
bitwise (it runs the same kernels on the same data; only its image tiles are
staged by cp.async instead of TMA), so that anything a call left in the
shared array would show up in the next one; one call is also checked against
the FP64 oracle.  This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2509_25924_gb300 as ofv
import synth

FP32_TOL = 1e-3  # the FP32 parity tolerance of the other GPU tests, in px
NDET_MIN = 1e-3  # pixels compared: oracle det / (Sxx + Syy)^2 at least this


def test_oversize_and_invalid_requests_are_rejected_before_any_device_work():
    p = ofv.ofv_default_params()
    with pytest.raises(ofv.OfvError) as ei:
        # 2048 x 2048 at FP32 storage needs ~108 MB of workspace; the
        # pointers are never dereferenced because the size check comes first
        ofv.ofv_compute_noalloc(2048, 2048, p, None, 16, 32, 48, 64, 0)
    assert ei.value.status == ofv.OFV_ERR_SHAPE
    assert "scratch" in ofv.ofv_last_error()
    with pytest.raises(ofv.OfvError) as ei:
        ofv.ofv_compute_noalloc(256, 256, ofv.ofv_default_params(path=ofv.OFV_PATH_PLAIN), None, 16, 32, 48, 64, 0)
    assert ei.value.status == ofv.OFV_ERR_UNSUPPORTED
    # the fields ofv_create range-checks are range-checked here too
    for field, bad in (("max_batch", -1), ("max_batch", 9), ("warm_start", -1), ("warm_start", 57),
                       ("tile_edge", 40)):
        q = ofv.ofv_default_params(**{field: bad})
        with pytest.raises(ofv.OfvError) as ei:
            ofv.ofv_compute_noalloc(256, 256, q, None, 16, 32, 48, 64, 0)
        assert ei.value.status == ofv.OFV_ERR_INVALID_ARG, field


def _lib():
    lib = ctypes.CDLL(ofv.lib_path)
    lib.ofv_compute_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ofv.Params)] + [ctypes.c_void_p] * 6
    lib.ofv_compute_noalloc.restype = ctypes.c_int
    return lib


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    torch.cuda.set_device(0)
    return torch


def _noalloc(torch, lib, H, W, p, I1, I2, w25=None):
    u = torch.full((H, W), float("nan"), device="cuda")
    v = torch.full((H, W), float("nan"), device="cuda")
    st = lib.ofv_compute_noalloc(H, W, ctypes.byref(p), None if w25 is None else w25.data_ptr(), I1.data_ptr(),
                                 I2.data_ptr(), u.data_ptr(), v.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == ofv.OFV_OK, ofv.ofv_last_error()
    return u, v


def _compute(torch, H, W, p, I1, I2, w25=None):
    h = ofv.ofv_create(H, W, p)
    try:
        if w25 is not None:
            ofv.ofv_set_prefilter(h, w25)
        u = torch.empty((H, W), device="cuda")
        v = torch.empty_like(u)
        ofv.ofv_compute(h, I1, I2, u, v)
        torch.cuda.synchronize()
        return u, v
    finally:
        ofv.ofv_destroy(h)


@pytest.mark.gpu
def test_noalloc_is_bitwise_ofv_compute_on_consecutive_calls():
    torch = _torch()
    lib = _lib()
    H, W = 1024, 1024
    frames = torch.from_numpy(synth.stream_frames(H, W, 3, seed=2)).to("cuda")
    p = ofv.ofv_default_params()
    for k in range(2):  # two calls in a row on different pairs
        I1, I2 = frames[k], frames[k + 1]
        u_ref, v_ref = _compute(torch, H, W, p, I1, I2)
        u, v = _noalloc(torch, lib, H, W, p, I1, I2)
        torch.cuda.synchronize()
        assert torch.equal(u, u_ref) and torch.equal(v, v_ref), f"call {k}"


@pytest.mark.gpu
def test_noalloc_matches_the_oracle():
    """One call against the FP64 oracle directly (not only through
    ofv_compute): FP32 storage, max |dV| <= 1e-3 px on the pixels the
    oracle finds well conditioned."""
    torch = _torch()
    lib = _lib()
    I1, I2, _, _ = synth.rankine_pair(256, 256, seed=1)
    p = ofv.ofv_default_params(input=ofv.OFV_IN_F32)
    u, v = _noalloc(torch, lib, 256, 256, p, torch.from_numpy(I1).cuda(), torch.from_numpy(I2).cuda())
    torch.cuda.synchronize()
    ou, ov, nd, _ = oracle.flow(I1.astype(np.float64), I2.astype(np.float64), oracle.Params(psl=2, kr=4, it=3),
                                diagnostics=True)
    m = nd >= NDET_MIN
    assert m.mean() > 0.99
    u, v = u.cpu().numpy(), v.cpu().numpy()
    err = max(np.abs(u - ou)[m].max(), np.abs(v - ov)[m].max())
    assert err <= FP32_TOL, f"max |dV| vs oracle {err:.3e}"


@pytest.mark.gpu
@pytest.mark.parametrize("storage,kr,edge", [(ofv.OFV_STORE_F16, 4, 0), (ofv.OFV_STORE_BF16, 4, 0),
                                             (ofv.OFV_STORE_F32, 12, 0), (ofv.OFV_STORE_F32, 4, 32)])
def test_noalloc_reduced_storage_and_large_radius(storage, kr, edge):
    """16-bit level storage (2 bytes per sample in the scratch layout), a
    radius above 10 (the tile kernel instead of the block kernel) and the
    alternative tile edge, bitwise against ofv_compute on two calls in a row."""
    torch = _torch()
    lib = _lib()
    H, W = 300, 420
    frames = torch.from_numpy(synth.stream_frames(H, W, 3, seed=9)).to("cuda")
    p = ofv.ofv_default_params(storage=storage, kernel_radius=kr, levels_psl=1 if kr > 10 else 2, tile_edge=edge)
    for k in range(2):
        u_ref, v_ref = _compute(torch, H, W, p, frames[k], frames[k + 1])
        u, v = _noalloc(torch, lib, H, W, p, frames[k], frames[k + 1])
        torch.cuda.synchronize()
        assert torch.equal(u, u_ref) and torch.equal(v, v_ref), f"call {k}"


@pytest.mark.gpu
def test_noalloc_prefilter_and_normalization():
    """A different shape, input type, local normalization and a pre-filter
    after the calls above, bitwise against ofv_compute."""
    torch = _torch()
    lib = _lib()
    I1, I2, _, _ = synth.rankine_pair(300, 200, seed=5)
    q = ofv.ofv_default_params(input=ofv.OFV_IN_F32, prefilter=1, norm_radius=1)
    w = np.zeros(25, np.float32)
    w[12] = 0.9
    w[7] = w[11] = w[13] = w[17] = 0.025
    wt = torch.from_numpy(w).to("cuda")
    t1 = torch.from_numpy(I1).to("cuda")
    t2 = torch.from_numpy(I2).to("cuda")
    u_ref, v_ref = _compute(torch, 300, 200, q, t1, t2, wt)
    u, v = _noalloc(torch, lib, 300, 200, q, t1, t2, wt)
    torch.cuda.synchronize()
    assert torch.equal(u, u_ref) and torch.equal(v, v_ref)
