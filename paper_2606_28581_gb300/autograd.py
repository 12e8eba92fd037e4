"""torch.autograd.Function over the CUDA rasterizer (training form a) and the shading (K7).

Forward runs project -> bin/sort -> rasterize in the CUDA library; backward runs
the hand-written adjoint (ss_rasterize_bwd).  Per pixel only T_final and the end
of the walk are saved; transmittances are recovered in the backward.

Inputs are FP32 master tensors.  With ``storage=torch.bfloat16`` the splat
attributes are stored in BF16 for the rasterizer (training form c) and the
gradients come back in FP32 with respect to those stored values, which the
optimiser applies to the masters.
"""
from __future__ import annotations

from typing import List, Sequence

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
                if frame.distortion:
                    flat.append(out.distort[i])
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
                if frame.distortion:
                    up[-1]["distort"] = c(next(it))
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
    Returns one dict per target: rgb, depth, normal, alpha, and distort when the frame was made
    with ``distortion=True`` (sun targets: depth, alpha)."""
    flat = _RenderFn.apply(frame, storage, means, scales, quats, opacity, rgb, dF, color)
    res, i = [], 0
    for t in frame.targets:
        if not t.sun:
            res.append(dict(rgb=flat[i], depth=flat[i + 1], normal=flat[i + 2], alpha=flat[i + 3]))
            i += 4
            if frame.distortion:
                res[-1]["distort"] = flat[i]
                i += 1
        else:
            res.append(dict(depth=flat[i], alpha=flat[i + 1]))
            i += 2
    return res


class _ShadeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, frame: Frame, opts, dF, La, *planes):
        V = frame.n_cams
        dev = La.device
        dFc = None if dF is None else dF.detach().float().contiguous()
        Lac = La.detach().float().contiguous()
        views, images, vis = [], [], []
        for c in range(V):
            rgb, depth, alpha, sd, sa = [t.detach().float().contiguous() for t in planes[5 * c:5 * c + 5]]
            images.append(torch.empty_like(rgb))
            vis.append(torch.empty_like(depth))
            views.append(dict(rgb=rgb, depth=depth, alpha=alpha, sun_depth=sd, sun_alpha=sa, image=images[c],
                              vis=vis[c]))
        L.shade_fwd(frame.cams, V, dFc, Lac, opts, L.shade_io_array(views))
        ctx.frame, ctx.opts, ctx.views, ctx.dF, ctx.La = frame, opts, views, dFc, Lac
        ctx.has_dF = dF is not None
        ctx.mark_non_differentiable(*vis)
        return tuple(images) + tuple(vis)

    @staticmethod
    def backward(ctx, *gouts):
        frame = ctx.frame
        V = frame.n_cams
        views, d_planes = [], []
        for c in range(V):
            v = dict(ctx.views[c])
            g = gouts[c]
            v["d_image"] = torch.zeros_like(v["rgb"]) if g is None else g.float().contiguous()
            d = dict(d_rgb=torch.zeros_like(v["rgb"]), d_depth=torch.zeros_like(v["depth"]),
                     d_alpha=torch.zeros_like(v["alpha"]), d_sun_depth=torch.zeros_like(v["sun_depth"]),
                     d_sun_alpha=torch.zeros_like(v["sun_alpha"]))
            v.update(d)
            views.append(v)
            d_planes += [d["d_rgb"], d["d_depth"], d["d_alpha"], d["d_sun_depth"], d["d_sun_alpha"]]
        d_La = torch.zeros_like(ctx.La)
        d_dF = torch.zeros(V, 2, 4, device=ctx.La.device) if ctx.has_dF else None
        L.shade_bwd(frame.cams, V, ctx.dF, ctx.La, ctx.opts, L.shade_io_array(views), d_La, d_dF)
        return (None, None, d_dF, d_La, *d_planes)


def shade(frame: Frame, targets: Sequence[dict], La, dF=None, opts=None) -> List[dict]:
    """Differentiable sun visibility and image formation (Sec. 3.1 Eq. image_formation) of every
    main view of ``frame`` (rendered with both passes) from the dicts ``render`` returned:
    I = (C A + c)(V + (1 - V) L_a).  La (V, 3) ambient light, dF (V, 2, 4) the camera deltas the
    render used (the sun position depends on them).  Returns one dict per view: image (3, H, W)
    and vis (H, W, not differentiable)."""
    V = frame.n_cams
    if len(frame.targets) != 2 * V:
        raise ValueError("shade needs a frame rendered with the main and the sun pass")
    planes = []
    for c in range(V):
        m, s = targets[c], targets[V + c]
        planes += [m["rgb"], m["depth"], m["alpha"], s["depth"], s["alpha"]]
    flat = _ShadeFn.apply(frame, opts if opts is not None else L.default_shade_opts(), dF, La, *planes)
    return [dict(image=flat[c], vis=flat[V + c]) for c in range(V)]


class _DepthNormalFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, frame: Frame, alpha_eps: float, dF, *planes):
        V = frame.n_cams
        dFc = None if dF is None else dF.detach().float().contiguous()
        views, normals = [], []
        for c in range(V):
            depth, alpha = [t.detach().float().contiguous() for t in planes[2 * c:2 * c + 2]]
            normals.append(torch.empty(3, *depth.shape, device=depth.device))
            views.append(dict(depth=depth, alpha=alpha, normal=normals[c]))
        L.depth_normal_fwd(frame.cams, V, dFc, alpha_eps, L.dnormal_io_array(views))
        ctx.frame, ctx.eps, ctx.views, ctx.dF, ctx.has_dF = frame, alpha_eps, views, dFc, dF is not None
        return tuple(normals)

    @staticmethod
    def backward(ctx, *gouts):
        frame = ctx.frame
        V = frame.n_cams
        views, d_planes = [], []
        for c in range(V):
            v = dict(ctx.views[c])
            g = gouts[c]
            v["d_normal"] = torch.zeros_like(v["normal"]) if g is None else g.float().contiguous()
            v["d_depth"] = torch.zeros_like(v["depth"])
            v["d_alpha"] = torch.zeros_like(v["alpha"])
            views.append(v)
            d_planes += [v["d_depth"], v["d_alpha"]]
        d_dF = torch.zeros(V, 2, 4, device=views[0]["depth"].device) if ctx.has_dF else None
        L.depth_normal_bwd(frame.cams, V, ctx.dF, ctx.eps, L.dnormal_io_array(views), d_dF)
        return (None, None, d_dF, *d_planes)


def depth_normal(frame: Frame, targets: Sequence[dict], dF=None, alpha_eps: float = 1e-3) -> List[torch.Tensor]:
    """Differentiable depth-gradient surface normal N (3, H, W) of every main view of ``frame``
    (Sec. 3.2 Eq. surface_normal) from the dicts ``render`` returned; with the rendered normal it
    gives the normal-consistency regulariser, e.g. (alpha - (normal * N).sum(0)).mean().  dF (V, 2, 4)
    the camera deltas the render used."""
    V = frame.n_cams
    planes = []
    for c in range(V):
        planes += [targets[c]["depth"], targets[c]["alpha"]]
    return list(_DepthNormalFn.apply(frame, float(alpha_eps), dF, *planes))
