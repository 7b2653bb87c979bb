"""Workspace hygiene and error paths on the GPU, without faulting it:
allocation failures injected through the library's allocator
(ofv_debug_fail_alloc) must give OFV_ERR_ALLOC and leak nothing, and a
workspace filled with NaN bytes (ofv_debug_poison) must not change any
result bitwise -- no output reads scratch that the call did not write."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2509_25924_gb300 as ofv  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_failed_create_allocations_leak_nothing():
    H, W = 512, 640
    p = ofv.ofv_default_params()
    h = ofv.ofv_create(H, W, p)  # warm: module loads and one-time allocations happen here
    ofv.ofv_destroy(h)
    base = _free_bytes()
    for n in (1, 2):
        ofv.ofv_debug_fail_alloc(n)
        try:
            try:
                h = ofv.ofv_create(H, W, p)
            except ofv.OfvError as e:
                assert e.status == ofv.OFV_ERR_ALLOC
            else:  # the n-th allocation came later than ofv_create
                ofv.ofv_destroy(h)
        finally:
            ofv.ofv_debug_fail_alloc(0)
        assert _free_bytes() >= base - (2 << 20)
    h = ofv.ofv_create(H, W, p)  # and the next create succeeds
    ofv.ofv_destroy(h)


def test_failed_workspace_growth_reports_alloc_and_the_handle_stays_usable():
    H, W = 256, 320
    F = synth.stream_frames(H, W, 4, seed=3)
    fr = torch.from_numpy(F).to(DEV)
    h = ofv.ofv_create(H, W, ofv.ofv_default_params(prefilter=1))
    try:
        u = torch.empty((H, W), device=DEV); v = torch.empty_like(u)
        ofv.ofv_compute(h, fr[0], fr[1], u, v)
        ref = (u.clone(), v.clone())
        g = torch.ones((H, W), device=DEV)
        calls = [
            ("host staging", lambda: ofv.ofv_compute_host(h, F[0], F[1], np.empty((H, W), np.float32),
                                                          np.empty((H, W), np.float32))),
            ("reverse mode", lambda: ofv.ofv_backward(h, fr[0], fr[1], g, g, torch.empty_like(u),
                                                      torch.empty_like(u))),
            ("batched", lambda: ofv.ofv_compute_batched(h, [(fr[0], fr[1], torch.empty_like(u),
                                                             torch.empty_like(u))])),
        ]
        for name, call in calls:
            ofv.ofv_debug_fail_alloc(1)
            try:
                with pytest.raises(ofv.OfvError) as ei:
                    call()
                assert ei.value.status == ofv.OFV_ERR_ALLOC, name
            finally:
                ofv.ofv_debug_fail_alloc(0)
            call()  # succeeds once memory is available
            torch.cuda.synchronize()
        ofv.ofv_compute(h, fr[0], fr[1], u, v)
        torch.cuda.synchronize()
        assert torch.equal(u, ref[0]) and torch.equal(v, ref[1])
    finally:
        ofv.ofv_destroy(h)


@pytest.mark.parametrize("path", [ofv.OFV_PATH_FUSED, ofv.OFV_PATH_PLAIN, ofv.OFV_PATH_TILE])
@pytest.mark.parametrize("storage", [ofv.OFV_STORE_F32, ofv.OFV_STORE_F16])
def test_poisoned_workspace_gives_bitwise_the_same_fields(path, storage):
    H, W, n = 200, 264, 6
    F = synth.stream_frames(H, W, n, seed=4)
    fr = torch.from_numpy(F).to(DEV)
    h = ofv.ofv_create(H, W, ofv.ofv_default_params(path=path, storage=storage, max_batch=2))
    try:
        out = []
        for poison in (False, True):
            if poison:
                ofv.ofv_debug_poison(h)
            us = torch.empty((n - 1, H, W), device=DEV); vs = torch.empty_like(us)
            ofv.ofv_compute_sequence(h, n, fr, H * W * 2, us, vs, H * W)
            u = torch.empty((H, W), device=DEV); v = torch.empty_like(u)
            if poison:
                ofv.ofv_debug_poison(h)
            ofv.ofv_compute(h, fr[2], fr[3], u, v)
            torch.cuda.synchronize()
            out.append((us, vs, u, v))
        for a, b in zip(out[0], out[1]):
            assert torch.isfinite(b).all() and torch.equal(a, b)
    finally:
        ofv.ofv_destroy(h)


def test_poisoned_workspace_for_the_batched_and_reverse_entry_points():
    H, W = 128, 160
    F = synth.stream_frames(H, W, 3, seed=5)
    fr = torch.from_numpy(F).to(DEV)
    h = ofv.ofv_create(H, W, ofv.ofv_default_params(prefilter=1))
    try:
        g = torch.randn((H, W), device=DEV, generator=torch.Generator(device=DEV).manual_seed(3))
        res = []
        for poison in (False, True):
            if poison:
                ofv.ofv_debug_poison(h)
            u = torch.empty((H, W), device=DEV); v = torch.empty_like(u)
            ofv.ofv_compute_batched(h, [(fr[0], fr[1], u, v)])
            if poison:
                ofv.ofv_debug_poison(h)
            g1 = torch.empty_like(u); g2 = torch.empty_like(u); gw = torch.empty(25, device=DEV)
            ofv.ofv_backward(h, fr[0], fr[1], g, g, g1, g2, gw)
            torch.cuda.synchronize()
            res.append((u, v, g1, g2, gw))
        assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
        for a, b in zip(res[0][2:], res[1][2:]):  # float atomics reorder the sums between runs
            assert torch.isfinite(b).all()
            assert float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(a)) <= 1e-4
    finally:
        ofv.ofv_destroy(h)
