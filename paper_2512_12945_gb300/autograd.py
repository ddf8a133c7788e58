"""torch.autograd.Function over the library's forward integration and its
adjoint kernel (slim_backward). The forward integrates every scan into an
emptied map and returns the extracted fields; the backward scatters the
incoming field gradients to the library's voxel index and runs the adjoint
once per scan, recomputing the (voxel, point) pairs instead of storing them.
With stored=True (closed set) the forward instead keeps each scan's pair
list (slim_record_pairs: 4 bytes per pair and per point) and the backward
reads it (slim_backward_pairs), with the same result; it exists to measure
what storing the pairs costs. Differentiable inputs: point coordinates
(sensor frame) and per-point class probabilities (closed-set soft counts)
or embeddings (open set)."""
from __future__ import annotations

import torch

from . import slim


class IntegrateFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, poses, stored, *tensors):
        pts, sem = tensors[0::2], tensors[1::2]
        m.reset()
        for p, s, pose in zip(pts, sem, poses):
            m.integrate(p.detach().contiguous(), pose, s.detach().contiguous())
        ext = m.extract(index=True)
        ctx.m, ctx.poses = m, poses
        # the stored form: each scan's pairs, recorded once the map holds
        # every scan (the voxel indices are final)
        ctx.pairs = [m.record_pairs(p.detach().contiguous(), pose)
                     for p, pose in zip(pts, poses)] if stored else None
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
        for k, (p, s, pose) in enumerate(zip(pts, sem, ctx.poses)):
            if ctx.pairs is not None:
                offs, vox = ctx.pairs[k]
                gsem, gxyz = m.backward_pairs(p.detach().contiguous(), pose, offs, vox, gD, gS)
            else:
                gsem, gxyz = m.backward(p.detach().contiguous(), pose, s.detach().contiguous(),
                                        gD, gS, gB)
            out += [gxyz, gsem]
        ctx.pairs = None
        return (None, None, None, *out)


def integrate(m, poses, pts, sem, stored=False):
    """Differentiable integration of scans (lists of tensors) into map m;
    stored=True keeps the pair lists for the backward (closed set)."""
    tensors = []
    for p, s in zip(pts, sem):
        tensors += [p, s]
    return IntegrateFn.apply(m, poses, bool(stored), *tensors)
