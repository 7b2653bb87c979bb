"""The allocation-free entry point, ofv_compute_noalloc.

It exists for callers that cannot call cudaMalloc: work recorded into a CUDA
graph by stream capture (which must not gain allocation nodes), host programs
whose device memory belongs to another allocator, and real-time loops that
forbid allocation once running.  Its workspace is a fixed device array inside
the library instead of a handle's allocation.  These tests call it through
the C ABI and compare it with the handle-based ofv_compute on consecutive
calls, so that anything a call left in the shared array would show up in
the next one.  This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import paper_2509_25924_gb300 as ofv
import synth

TOL = 1e-3  # the FP32 parity tolerance of the other GPU tests, in px


def test_oversize_requests_are_rejected_before_any_device_work():
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


@pytest.mark.gpu
def test_noalloc_matches_ofv_compute_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    lib = ctypes.CDLL(ofv.lib_path)
    lib.ofv_compute_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ofv.Params)] + [ctypes.c_void_p] * 6
    lib.ofv_compute_noalloc.restype = ctypes.c_int

    H, W = 1024, 1024
    frames = torch.from_numpy(synth.stream_frames(H, W, 3, seed=2)).to(dev)
    p = ofv.ofv_default_params()
    stream = torch.cuda.current_stream()
    h = ofv.ofv_create(H, W, p)
    try:
        for k in range(2):  # two calls in a row on different pairs
            I1, I2 = frames[k], frames[k + 1]
            u_ref = torch.empty((H, W), dtype=torch.float32, device=dev)
            v_ref = torch.empty_like(u_ref)
            ofv.ofv_compute(h, I1, I2, u_ref, v_ref, stream)
            u = torch.full((H, W), float("nan"), device=dev)
            v = torch.full((H, W), float("nan"), device=dev)
            st = lib.ofv_compute_noalloc(H, W, ctypes.byref(p), None, I1.data_ptr(), I2.data_ptr(), u.data_ptr(),
                                         v.data_ptr(), stream.cuda_stream)
            assert st == ofv.OFV_OK, ofv.ofv_last_error()
            torch.cuda.synchronize()
            assert torch.isfinite(u).all() and torch.isfinite(v).all()
            du = (u - u_ref).abs().max().item()
            dv = (v - v_ref).abs().max().item()
            assert du <= TOL and dv <= TOL, f"call {k}: max |du|={du:.3e} |dv|={dv:.3e}"
    finally:
        ofv.ofv_destroy(h)

    # a different shape, input type and a pre-filter after the calls above
    I1, I2, _, _ = synth.rankine_pair(300, 200, seed=5)
    q = ofv.ofv_default_params(input=ofv.OFV_IN_F32, prefilter=1, norm_radius=1)
    w = np.zeros(25, np.float32)
    w[12] = 0.9
    w[7] = w[11] = w[13] = w[17] = 0.025
    wt = torch.from_numpy(w).to(dev)
    t1 = torch.from_numpy(I1).to(dev)
    t2 = torch.from_numpy(I2).to(dev)
    h = ofv.ofv_create(300, 200, q)
    try:
        ofv.ofv_set_prefilter(h, wt)
        u_ref = torch.empty((300, 200), device=dev)
        v_ref = torch.empty_like(u_ref)
        ofv.ofv_compute(h, t1, t2, u_ref, v_ref)
        u = torch.empty_like(u_ref)
        v = torch.empty_like(u_ref)
        st = lib.ofv_compute_noalloc(300, 200, ctypes.byref(q), wt.data_ptr(), t1.data_ptr(), t2.data_ptr(),
                                     u.data_ptr(), v.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert st == ofv.OFV_OK, ofv.ofv_last_error()
        torch.cuda.synchronize()
        assert (u - u_ref).abs().max().item() <= TOL and (v - v_ref).abs().max().item() <= TOL
    finally:
        ofv.ofv_destroy(h)
