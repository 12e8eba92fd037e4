"""Batched multi-view training step in CUDA graphs (training form b).

All views and their sun views form one frame.  One step is: camera assembly +
projection (K1), one shared height sort + binning of every target (K2), ONE
persistent forward launch over every (target, tile) item (K3), ONE persistent
backward launch (K4) and the projection adjoint (K5).  The step is captured once
as two CUDA graphs (forward part, backward part) and replayed; the intersection
capacity is fixed at capture and an overflow is reported through the workspace
status block, which the host reads after a replay (``check``).  From host
buffers (``replay_from_host``) the upstream gradients are copied on a side
stream while the forward part runs, and only the backward part waits for them.

The autotuner times the candidate tile shapes (each with the kernels' own staging,
which the options' batch of 256 selects) on the actual workload and caches the
winner per (GPU, workload) in a JSON file.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Optional, Sequence

import torch

from . import _lib as L
from .frame import Frame, Outputs, grads_struct

# (tile_w, tile_h, batch, pixels per thread)
TILE_CANDIDATES = [(16, 16, 256, 4), (32, 8, 256, 4), (8, 32, 256, 4), (32, 16, 256, 4), (16, 32, 256, 4)]


def _opts(c):
    tw, th, b, ppt = c
    return L.default_opts(tile_w=tw, tile_h=th, batch=b, pixels_per_thread=ppt, persistent=1)


class BatchedStep:
    """One training step (forward + backward) over every target of a frame.

    ``splats``: dict of planar storage tensors [C, n_pad] (fp32 or bf16): means, scales,
    quats, opacity, rgb.  ``dF`` (V, 2, 4), ``color`` (V, 3, 4) fp32.  ``upstream``: one
    dict of upstream gradient planes per target (with ``distortion``, a main target's dict may
    hold the distortion's upstream under "distort").  Gradients go to ``grads`` (fp32 [C, n_pad]),
    ``d_dF`` and ``d_color``; they are zeroed at the start of each step."""

    def __init__(self, cameras: Sequence, splats: dict, n: int, dF, color, upstream: Sequence[dict],
                 passes: int = L.SS_PASS_MAIN | L.SS_PASS_SUN, opts: Optional[L.ss_raster_opts] = None,
                 capacity_slack: float = 1.10, capacity: Optional[int] = None, device="cuda",
                 distortion: bool = False):
        self.opts = opts if opts is not None else L.default_opts(persistent=1)
        self.frame = Frame(cameras, passes, self.opts, device=device, distortion=distortion)
        self.tensors = splats
        self.n = int(n)
        self.splats = L.make_splats(splats["means"], splats["scales"], splats["quats"], splats["opacity"],
                                    splats["rgb"], n)
        self.dF, self.color, self.upstream = dF, color, list(upstream)
        n_pad = int(splats["means"].shape[-1])
        z = lambda c: torch.zeros(c, n_pad, device=device, dtype=torch.float32)
        self.grads = dict(means=z(3), scales=z(2), quats=z(4), opacity=z(1), rgb=z(3))
        V = self.frame.n_cams
        self.d_dF = torch.zeros(V, 2, 4, device=device)
        self.d_color = torch.zeros(V, 3, 4, device=device)
        self.out = Outputs(self.frame.targets, self.frame.device, distortion)
        self._io_f = self.out.io_array()
        self._io_b = self.out.io_array(self.upstream)
        self._g = grads_struct(self.grads)
        self.graph = None
        self._copy_stream = None
        # size the intersection capacity with one synchronised eager run
        needed = self.frame.project_and_bin(self.splats, self.dF, self.color, sync=True)
        cap = capacity if capacity is not None else max(1 << 16, int(needed * capacity_slack) + 4096)
        self.frame.ensure_workspace(self.splats, cap)

    # ------------------------------------------------------------------ phases
    def project(self, stream=None):
        f = self.frame
        L.project_splats(self.splats, f.cams, f.n_cams, f.passes, self.dF, self.color, f.opts, f.ws, f.ws_bytes,
                         f.capacity,
                         stream)

    def bin(self, stream=None):
        f = self.frame
        L.bin_and_sort(self.splats, f.cams, f.n_cams, f.passes, f.opts, f.ws, f.ws_bytes, f.capacity,
                       sync_needed=False, stream=stream)

    def forward(self, stream=None):
        f = self.frame
        L.rasterize_fwd(self.splats, f.cams, f.n_cams, f.passes, f.opts, self._io_f, f.ws, f.ws_bytes,
                        f.capacity, stream)

    def backward_pixels(self, stream=None):
        f = self.frame
        L.rasterize_bwd(self.splats, f.cams, f.n_cams, f.passes, f.opts, self._io_b, None, None,
                        self.d_color, f.ws, f.ws_bytes, f.capacity, stream)

    def backward_project(self, stream=None):
        f = self.frame
        L.project_bwd(self.splats, f.cams, f.n_cams, f.passes, f.opts, self._g, self.d_dF, self.d_color, f.ws,
                      f.ws_bytes,
                      f.capacity, stream)

    def zero_grads(self):
        for g in self.grads.values():
            g.zero_()
        self.d_dF.zero_()
        self.d_color.zero_()

    def forward_part(self, stream=None):
        self.project(stream)
        self.bin(stream)
        self.forward(stream)

    def backward_part(self, stream=None):
        self.zero_grads()
        self.backward_pixels(stream)
        self.backward_project(stream)

    def step_eager(self, stream=None):
        self.forward_part(stream)
        self.backward_part(stream)

    # ------------------------------------------------------------------ graph
    def capture(self):
        """Capture one step as two CUDA graphs (after an eager warm-up run): the forward part
        (projection, binning, forward) and the backward part (gradient zeroing, backward,
        projection adjoint)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step_eager()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        gf, gb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(gf):
            self.forward_part()
        with torch.cuda.graph(gb, pool=gf.pool()):
            self.backward_part()
        torch.cuda.synchronize()
        self.graph = (gf, gb)
        return self.graph

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph[0].replay()
        self.graph[1].replay()

    def replay_from_host(self, h_splats: dict, h_dF, h_color, h_upstream: Sequence[dict], h_grads: dict,
                         h_d_dF=None, h_d_color=None):
        """One step from pinned host buffers: splats, camera deltas and colour corrections are
        copied in, the upstream gradient planes follow on a side stream while the forward part
        runs, the backward part waits for them, and the gradients are copied out (into
        ``h_grads`` and the optional ``h_d_dF`` / ``h_d_color``).  Asynchronous: synchronise the
        current stream before reading the host results."""
        if self.graph is None:
            self.capture()
        cur = torch.cuda.current_stream()
        if self._copy_stream is None:
            self._copy_stream = torch.cuda.Stream()
        side = self._copy_stream
        # the upstream planes may be overwritten once the work already on the current stream
        # (the previous step's backward) is done; they need not wait for this step's splat copies
        prior = torch.cuda.Event()
        prior.record(cur)
        for k, t in self.tensors.items():
            t.copy_(h_splats[k], non_blocking=True)
        self.dF.copy_(h_dF, non_blocking=True)
        self.color.copy_(h_color, non_blocking=True)
        side.wait_event(prior)
        with torch.cuda.stream(side):
            for du, hu in zip(self.upstream, h_upstream):
                for k in du:
                    du[k].copy_(hu[k], non_blocking=True)
        self.graph[0].replay()
        cur.wait_stream(side)
        self.graph[1].replay()
        for k, v in self.grads.items():
            h_grads[k].copy_(v, non_blocking=True)
        if h_d_dF is not None:
            h_d_dF.copy_(self.d_dF, non_blocking=True)
        if h_d_color is not None:
            h_d_color.copy_(self.d_color, non_blocking=True)

    def check(self):
        """Synchronise and read the status block: (status, needed, walked, flags).  ``walked``
        is 0 unless the last forward counted its pairs (``count_walked``)."""
        st, needed, _, walked, flags = self.frame.status()
        return st, needed, walked, flags

    def count_walked(self, stream=None) -> int:
        """Runs the forward part once eagerly with the walked-pair count (outside the graphs,
        which run without it) and returns the number of (pixel, splat) pairs walked: those with
        alpha >= alpha_min up to and including each pixel's stopping one."""
        f = self.frame
        o = L.ss_raster_opts.from_buffer_copy(f.opts)
        o.count_pairs = 1
        self.project(stream)
        self.bin(stream)
        L.rasterize_fwd(self.splats, f.cams, f.n_cams, f.passes, o, self._io_f, f.ws, f.ws_bytes, f.capacity, stream)
        st, _, walked, _ = self.check()
        if st != L.SS_OK:
            raise L.SatSplatError(st, "count_walked")
        return walked

    @property
    def main_pixels(self) -> int:
        return sum(t.width * t.height for t in self.frame.targets if not t.sun)

    @property
    def sun_pixels(self) -> int:
        return sum(t.width * t.height for t in self.frame.targets if t.sun)


# ------------------------------------------------------------------------------ autotuner
def _cache_path() -> str:
    base = os.environ.get("SATSPLAT_AUTOTUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "satsplat", "autotune.json")
    return base


def workload_key(cameras: Sequence, n: int, dtype, passes: int) -> str:
    h = hashlib.sha256()
    h.update(f"warp-items|{n}|{dtype}|{passes}".encode())
    for c in cameras:
        h.update(f"{c.width}x{c.height}|{c.shadow_w}x{c.shadow_h}".encode())
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return f"{name}|{h.hexdigest()[:16]}"


def autotune(make_step, key: str, candidates=TILE_CANDIDATES, warmup: int = 1, iters: int = 3,
             use_cache: bool = True, log=None):
    """Time ``make_step(opts)`` (a BatchedStep) for each (tile_w, tile_h, batch, ppt) candidate with
    persistent launches and return the fastest options.  Results are cached by ``key``."""
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except Exception:
            cache = {}
    if use_cache and key in cache and len(cache[key].get("best", ())) == 4:
        return _opts(cache[key]["best"]), cache[key]
    results = {}
    for cand in candidates:
        opts = _opts(cand)
        step = make_step(opts)
        for _ in range(warmup):
            step.step_eager()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times = []
        for _ in range(iters):
            ev0.record()
            step.step_eager()
            ev1.record()
            ev1.synchronize()
            times.append(ev0.elapsed_time(ev1))
        times.sort()
        name = "x".join(str(v) for v in cand)
        results[name] = times[len(times) // 2]
        if log:
            log(f"autotune tile {cand[0]}x{cand[1]} batch {cand[2]} ppt {cand[3]}: {results[name]:.3f} ms")
        del step
        torch.cuda.empty_cache()
    best = [int(v) for v in min(results, key=results.get).split("x")]
    entry = {"best": best, "ms": results}
    if use_cache:
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            cache[key] = entry
            json.dump(cache, open(path, "w"), indent=1)
        except OSError:
            pass
    return _opts(best), entry
