"""torch.autograd wrapper of the estimator.

``flow_fn(flow, I1, I2, w25=None)`` returns (u, v) like ``Flow.__call__`` and
records a node whose backward calls ``ofv_backward``: gradients reach the
two frames (FP32 input) and the 5x5 pre-filter weights.  Both passes run in
the library's CUDA kernels; this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import Flow, ofv_backward, ofv_set_prefilter, OFV_IN_F32


class FlowFunction(torch.autograd.Function):
    """u, v = FlowFunction.apply(I1, I2, w25, flow).  w25 is a 5x5 float32
    CUDA tensor (None when the handle's pre-filter is off)."""

    @staticmethod
    def forward(ctx, I1, I2, w25, flow: Flow):
        if w25 is not None:
            ofv_set_prefilter(flow.h, w25.detach().contiguous().float().reshape(25))
        u, v = flow(I1, I2)
        ctx.flow = flow
        ctx.save_for_backward(I1, I2, w25)
        return u, v

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, gu, gv):
        I1, I2, w25 = ctx.saved_tensors
        flow: Flow = ctx.flow
        H, W = flow.H, flow.W
        dev = I1.device
        gu = torch.zeros((H, W), dtype=torch.float32, device=dev) if gu is None else gu.float().contiguous()
        gv = torch.zeros((H, W), dtype=torch.float32, device=dev) if gv is None else gv.float().contiguous()
        if w25 is not None:  # the handle may have run with other weights since forward
            ofv_set_prefilter(flow.h, w25.detach().contiguous().float().reshape(25))
        gI1 = torch.empty((H, W), dtype=torch.float32, device=dev)
        gI2 = torch.empty((H, W), dtype=torch.float32, device=dev)
        gw = torch.empty(25, dtype=torch.float32, device=dev) if w25 is not None else None
        ofv_backward(flow.h, I1, I2, gu, gv, gI1, gI2, gw)
        f = flow.params.input == OFV_IN_F32
        return (gI1 if f and ctx.needs_input_grad[0] else None,
                gI2 if f and ctx.needs_input_grad[1] else None,
                gw.view(5, 5).to(w25.dtype) if w25 is not None and ctx.needs_input_grad[2] else None,
                None)


def flow_fn(flow: Flow, I1, I2, w25=None):
    """Differentiable (u, v) of the pair (I1, I2) on the handle ``flow``."""
    return FlowFunction.apply(I1, I2, w25, flow)


_handles: dict = {}


def apply(I1, I2, prefilter_w=None, params=None):
    """Differentiable (u, v) of (I1, I2) for estimator parameters ``params``
    (an ofv_params structure, a dict of its fields, or None for the
    defaults; input type and pre-filter follow the arguments).  Handles are
    created on first use per (device, shape, parameters) and kept."""
    from . import ofv_default_params, Params, OFV_IN_F32, OFV_IN_U16, OFV_IN_U8
    kw = {}
    if isinstance(params, Params):
        kw = {name: getattr(params, name) for name, _ in Params._fields_}
    elif params:
        kw = dict(params)
    kw["input"] = {torch.float32: OFV_IN_F32, torch.uint8: OFV_IN_U8}.get(I1.dtype, OFV_IN_U16)
    kw["prefilter"] = 0 if prefilter_w is None else 1
    H, W = I1.shape[-2], I1.shape[-1]
    key = (I1.device.index, H, W, tuple(sorted(kw.items())))
    flow = _handles.get(key)
    if flow is None:
        with torch.cuda.device(I1.device):
            flow = Flow(H, W, ofv_default_params(**kw))
        _handles[key] = flow
    return FlowFunction.apply(I1, I2, prefilter_w, flow)
