"""Frame: one set of (cameras, passes, options) with its device workspace and outputs.

A thin orchestration layer over the C ABI: it allocates the caller-owned
buffers with PyTorch and calls ``ss_project_splats -> ss_bin_and_sort ->
ss_rasterize_fwd`` and ``ss_rasterize_bwd``.  All arithmetic runs in the CUDA
library.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import torch

from . import _lib as L


@dataclasses.dataclass
class Target:
    cam: int
    sun: bool
    width: int
    height: int


class Outputs:
    """Planes of every render target: rgb (3,H,W) / depth (H,W) / normal (3,H,W) / alpha
    (H,W) and the saved state T_final (H,W) f32 and last (H,W) int32 (uint32 bits).  With
    ``distortion`` the main targets also get the distortion plane distort (H,W)."""

    def __init__(self, targets: Sequence[Target], device, distortion: bool = False):
        self.rgb, self.depth, self.normal, self.alpha, self.T_final, self.last = [], [], [], [], [], []
        self.distort = []
        for t in targets:
            H, W = t.height, t.width
            f = lambda *s: torch.empty(*s, device=device, dtype=torch.float32)
            self.rgb.append(None if t.sun else f(3, H, W))
            self.depth.append(f(H, W))
            self.normal.append(None if t.sun else f(3, H, W))
            self.alpha.append(f(H, W))
            self.T_final.append(f(H, W))
            self.last.append(torch.empty(H, W, device=device, dtype=torch.int32))
            self.distort.append(f(H, W) if distortion and not t.sun else None)

    def io_array(self, upstream: Optional[dict] = None):
        n = len(self.depth)
        arr = (L.ss_target_io * n)()
        for i in range(n):
            a = arr[i]
            a.rgb, a.depth, a.normal, a.alpha = (L.ptr(self.rgb[i]), L.ptr(self.depth[i]),
                                                 L.ptr(self.normal[i]), L.ptr(self.alpha[i]))
            a.T_final, a.last = L.ptr(self.T_final[i]), L.ptr(self.last[i])
            a.distort = L.ptr(self.distort[i])
            if upstream is not None:
                u = upstream[i]
                a.d_rgb = L.ptr(u.get("rgb"))
                a.d_depth = L.ptr(u.get("depth"))
                a.d_normal = L.ptr(u.get("normal"))
                a.d_alpha = L.ptr(u.get("alpha"))
                a.d_distort = L.ptr(u.get("distort"))
        return arr


def pad_planar(x: torch.Tensor, n_pad: int) -> torch.Tensor:
    """[C, n] -> contiguous [C, n_pad] (zero padded)."""
    if x.dim() == 1:
        x = x[None]
    if x.shape[-1] == n_pad and x.is_contiguous():
        return x
    out = torch.zeros(x.shape[0], n_pad, device=x.device, dtype=x.dtype)
    out[:, : x.shape[-1]] = x
    return out


def n_pad_of(n: int) -> int:
    return max(8, (n + 7) // 8 * 8)


class Frame:
    """``distortion``: the main targets' outputs include the distortion plane."""

    def __init__(self, cameras: Sequence, passes: int = L.SS_PASS_MAIN, opts: Optional[L.ss_raster_opts] = None,
                 capacity: Optional[int] = None, device="cuda", distortion: bool = False):
        self.cam_objs = list(cameras)
        self.cams = L.make_cameras(self.cam_objs)
        self.n_cams = len(self.cam_objs)
        self.passes = int(passes)
        self.opts = opts if opts is not None else L.default_opts()
        self.device = torch.device(device)
        self.distortion = bool(distortion)
        self.targets: List[Target] = []
        if self.passes & L.SS_PASS_MAIN:
            self.targets += [Target(i, False, c.width, c.height) for i, c in enumerate(self.cam_objs)]
        if self.passes & L.SS_PASS_SUN:
            self.targets += [Target(i, True, c.shadow_w, c.shadow_h) for i, c in enumerate(self.cam_objs)]
        self.capacity = capacity
        self.ws = None
        self.ws_bytes = 0
        self.needed = None
        self._ws_key = None

    # -------------------------------------------------------------- workspace
    def ensure_workspace(self, splats: L.ss_splats, capacity: int):
        key = (int(splats.n), int(splats.n_pad), int(splats.dtype), int(capacity))
        if self.ws is not None and self._ws_key == key:
            return
        nbytes = L.workspace_size(splats, self.cams, self.n_cams, self.passes, self.opts, capacity)
        self.ws = None
        self.ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        self.ws_bytes = nbytes
        self.capacity = int(capacity)
        self._ws_key = key

    def default_capacity(self, n: int) -> int:
        px = sum(t.width * t.height for t in self.targets)
        tiles = px / float(self.opts.tile_w * self.opts.tile_h)
        return int(min(2 ** 31 - 1, max(1 << 16, 6 * n * len(self.targets), 600 * tiles)))

    # -------------------------------------------------------------- passes
    def project_and_bin(self, splats: L.ss_splats, dF: Optional[torch.Tensor], color=None, sync: bool = True,
                        stream=None) -> int:
        """Project, bin and sort.  With ``sync`` the intersection count is read back and the
        workspace grown and the frame re-run when it did not fit; returns the count."""
        cap = self.capacity if self.capacity is not None else self.default_capacity(int(splats.n))
        for _ in range(3):
            self.ensure_workspace(splats, cap)
            L.project_splats(splats, self.cams, self.n_cams, self.passes, dF, color, self.opts, self.ws,
                             self.ws_bytes, self.capacity, stream)
            st, needed = L.bin_and_sort(splats, self.cams, self.n_cams, self.passes, self.opts, self.ws,
                                        self.ws_bytes, self.capacity, sync_needed=sync, stream=stream)
            if not sync:
                return -1
            self.needed = needed
            if st == L.SS_OK:
                return needed
            cap = int(needed * 1.15) + 1024
        raise L.SatSplatError(L.SS_ERR_CAPACITY, "Frame.project_and_bin")

    def forward(self, splats: L.ss_splats, dF=None, color=None, out: Optional[Outputs] = None,
                sync: bool = True, stream=None) -> Outputs:
        self.project_and_bin(splats, dF, color, sync=sync, stream=stream)
        out = out if out is not None else Outputs(self.targets, self.device, self.distortion)
        io = out.io_array()
        L.rasterize_fwd(splats, self.cams, self.n_cams, self.passes, self.opts, io, self.ws,
                        self.ws_bytes, self.capacity, stream)
        return out

    def rasterize(self, splats: L.ss_splats, out: Outputs, stream=None):
        io = out.io_array()
        L.rasterize_fwd(splats, self.cams, self.n_cams, self.passes, self.opts, io, self.ws,
                        self.ws_bytes, self.capacity, stream)

    def backward(self, splats: L.ss_splats, out: Outputs, upstream: Sequence[dict], grads: dict,
                 d_dF=None, d_color=None, stream=None):
        """Accumulate gradients into ``grads`` (dict of fp32 [C, n_pad] tensors: means,
        scales, quats, opacity, rgb) and into d_dF [V,2,4] / d_color [V,3,4]."""
        io = out.io_array(upstream)
        g = grads_struct(grads)
        L.rasterize_bwd(splats, self.cams, self.n_cams, self.passes, self.opts, io, g, d_dF,
                        d_color, self.ws, self.ws_bytes, self.capacity, stream)

    def backward_pixels(self, splats: L.ss_splats, out: Outputs, upstream: Sequence[dict], d_color=None,
                        stream=None):
        """Per-pixel adjoint only (K4); finish with :meth:`backward_project`."""
        io = out.io_array(upstream)
        L.rasterize_bwd(splats, self.cams, self.n_cams, self.passes, self.opts, io, None, None,
                        d_color, self.ws, self.ws_bytes, self.capacity, stream)

    def backward_project(self, splats: L.ss_splats, grads: dict, d_dF=None, d_color=None, stream=None):
        """Projection adjoint (K5) of the records left by :meth:`backward_pixels`."""
        L.project_bwd(splats, self.cams, self.n_cams, self.passes, self.opts, grads_struct(grads), d_dF, d_color,
                      self.ws, self.ws_bytes, self.capacity, stream)

    def status(self, stream=None):
        return L.frame_status(self.ws, self.ws_bytes, stream)


def grads_struct(grads: dict) -> L.ss_splat_grads:
    g = L.ss_splat_grads()
    g.means, g.scales, g.quats = L.ptr(grads["means"]), L.ptr(grads["scales"]), L.ptr(grads["quats"])
    g.opacity, g.rgb = L.ptr(grads["opacity"]), L.ptr(grads["rgb"])
    g.n_pad = int(grads["means"].shape[-1])
    return g


def zero_grads(n_pad: int, device) -> dict:
    z = lambda c: torch.zeros(c, n_pad, device=device, dtype=torch.float32)
    return dict(means=z(3), scales=z(2), quats=z(4), opacity=z(1), rgb=z(3))
