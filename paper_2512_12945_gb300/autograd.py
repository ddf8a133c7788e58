"""torch.autograd.Function over the library's forward integration and its
adjoint kernel (slim_backward). The forward integrates every scan into an
emptied map and returns the extracted fields; the backward scatters the
incoming field gradients to the library's voxel index and runs the adjoint
once per scan, recomputing the (voxel, point) pairs instead of storing them.
Differentiable inputs: point coordinates (sensor frame) and per-point class
probabilities (closed-set soft counts) or embeddings (open set)."""
from __future__ import annotations

import torch

from . import slim


class IntegrateFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, poses, *tensors):
        pts, sem = tensors[0::2], tensors[1::2]
        m.reset()
        for p, s, pose in zip(pts, sem, poses):
            m.integrate(p.detach().contiguous(), pose, s.detach().contiguous())
        ext = m.extract(index=True)
        ctx.m, ctx.poses = m, poses
        ctx.index = ext["index"].long()
        ctx.save_for_backward(*tensors)
        ctx.mark_non_differentiable(ext["W"], ext["ijk"])
        if m.mode == slim.SLIM_OPEN:
            return ext["D"], ext["W"], ext["sem"], ext["beta"], ext["ijk"]
        return ext["D"], ext["W"], ext["sem"], ext["ijk"]

    @staticmethod
    def backward(ctx, *grads):
        m = ctx.m
        tensors = ctx.saved_tensors
        pts, sem = tensors[0::2], tensors[1::2]
        idx = ctx.index
        size = int(idx.max().item()) + 1 if idx.numel() else 1
        dev = idx.device

        def dense(g, width=None):
            shape = (size,) if width is None else (size, width)
            out = torch.zeros(shape, dtype=torch.float32, device=dev)
            if g is not None and idx.numel():
                out[idx] = g.to(torch.float32)
            return out

        gD = dense(grads[0])
        gS = dense(grads[2], m.width)
        gB = dense(grads[3], m.width) if m.mode == slim.SLIM_OPEN else None
        out = []
        for p, s, pose in zip(pts, sem, ctx.poses):
            gsem, gxyz = m.backward(p.detach().contiguous(), pose, s.detach().contiguous(),
                                    gD, gS, gB)
            out += [gxyz, gsem]
        return (None, None, *out)


def integrate(m, poses, pts, sem):
    """Differentiable integration of scans (lists of tensors) into map m."""
    tensors = []
    for p, s in zip(pts, sem):
        tensors += [p, s]
    return IntegrateFn.apply(m, poses, *tensors)
