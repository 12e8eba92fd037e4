"""torch.autograd.Function over the CUDA rasterizer (training form a).

Forward runs project -> bin/sort -> rasterize in the CUDA library; backward runs
the hand-written adjoint (ss_rasterize_bwd).  Per pixel only T_final and the end
of the walk are saved; transmittances are recovered in the backward.

Inputs are FP32 master tensors.  With ``storage=torch.bfloat16`` the splat
attributes are stored in BF16 for the rasterizer (training form c) and the
gradients come back in FP32 with respect to those stored values, which the
optimiser applies to the masters.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import torch

from . import _lib as L
from .frame import Frame, n_pad_of, pad_planar, zero_grads


def _store(x: torch.Tensor, n_pad: int, dtype) -> torch.Tensor:
    x = x.detach()
    if x.dim() == 1:
        x = x[None]
    return pad_planar(x.to(dtype).contiguous(), n_pad)


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, frame: Frame, storage, means, scales, quats, opacity, rgb, dF, color):
        n = int(means.shape[-1])
        n_pad = n_pad_of(n)
        store = [_store(t, n_pad, storage) for t in (means, scales, quats, opacity, rgb)]
        splats = L.make_splats(*store, n)
        dFc = None if dF is None else dF.detach().float().contiguous()
        colc = None if color is None else color.detach().float().contiguous()
        out = frame.forward(splats, dFc, colc)
        frame._generation = getattr(frame, "_generation", 0) + 1
        ctx.frame, ctx.store, ctx.out, ctx.n, ctx.n_pad = frame, store, out, n, n_pad
        ctx.generation = frame._generation
        ctx.dF, ctx.color = dFc, colc
        ctx.has_dF, ctx.has_color = dF is not None, color is not None
        flat = []
        for i, t in enumerate(frame.targets):
            if not t.sun:
                flat += [out.rgb[i], out.depth[i], out.normal[i], out.alpha[i]]
            else:
                flat += [out.depth[i], out.alpha[i]]
        return tuple(flat)

    @staticmethod
    def backward(ctx, *gouts):
        frame: Frame = ctx.frame
        splats = L.make_splats(*ctx.store, ctx.n)
        if getattr(frame, "_generation", 0) != ctx.generation:
            # the frame's workspace was reused by a later forward: rebuild this frame's lists
            frame.project_and_bin(splats, ctx.dF, ctx.color)
        up = []
        it = iter(gouts)
        c = lambda g: None if g is None else g.float().contiguous()
        for t in frame.targets:
            if not t.sun:
                up.append(dict(rgb=c(next(it)), depth=c(next(it)), normal=c(next(it)), alpha=c(next(it))))
            else:
                up.append(dict(depth=c(next(it)), alpha=c(next(it))))
        dev = ctx.store[0].device
        grads = zero_grads(ctx.n_pad, dev)
        d_dF = torch.zeros(frame.n_cams, 2, 4, device=dev) if ctx.has_dF else None
        d_color = torch.zeros(frame.n_cams, 3, 4, device=dev) if ctx.has_color else None
        frame.backward(splats, ctx.out, up, grads, d_dF=d_dF, d_color=d_color)
        n = ctx.n
        return (None, None, grads["means"][:, :n], grads["scales"][:, :n], grads["quats"][:, :n],
                grads["opacity"][0, :n], grads["rgb"][:, :n], d_dF, d_color)


def render(frame: Frame, means, scales, quats, opacity, rgb, dF=None, color=None,
           storage=torch.float32) -> List[dict]:
    """Differentiable render of every target of ``frame``.

    means (3, N), scales (2, N), quats (4, N) (w, x, y, z), opacity (N,), rgb (3, N): FP32.
    dF (V, 2, 4) camera deltas and color (V, 3, 4) [C | c], optional.
    Returns one dict per target: rgb, depth, normal, alpha (sun targets: depth, alpha)."""
    flat = _RenderFn.apply(frame, storage, means, scales, quats, opacity, rgb, dF, color)
    res, i = [], 0
    for t in frame.targets:
        if not t.sun:
            res.append(dict(rgb=flat[i], depth=flat[i + 1], normal=flat[i + 2], alpha=flat[i + 3]))
            i += 4
        else:
            res.append(dict(depth=flat[i], alpha=flat[i + 1]))
            i += 2
    return res
