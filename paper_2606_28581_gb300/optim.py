"""SplatOptimizer: the splats' raw parameters, Adam moments and rasterizer storage under a fixed
splat budget, updated by the fused Adam step and the 3DGS-MCMC relocation of the CUDA library.

Memory is allocated once for the budget ``cap`` (planar [C, n_pad(cap)] arrays), so growth never
reallocates: the active count ``n`` moves within it.  All arithmetic runs in the CUDA library
(``ss_adam_step``, ``ss_mcmc_relocate``); this class only owns the buffers.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import _lib as L
from .frame import n_pad_of

ROWS = dict(means=3, log_scales=2, quats=4, logit_opacity=1, rgb=3)
STORE_ROWS = dict(means=3, scales=2, quats=4, opacity=1, rgb=3)


class SplatOptimizer:
    """``means`` (3, n), ``scales`` (2, n) > 0, ``quats`` (4, n), ``opacity`` (n,) in (0, 1),
    ``rgb`` (3, n): activated initial values.  ``storage``: the dtype the rasterizer reads."""

    def __init__(self, means, scales, quats, opacity, rgb, cap: int, storage=torch.bfloat16,
                 adam: Optional[L.ss_adam_opts] = None, mcmc: Optional[L.ss_mcmc_opts] = None, seed: int = 0,
                 device="cuda"):
        n = int(means.shape[-1])
        if not (0 < n <= cap):
            raise ValueError("need 0 < n <= cap")
        self.cap, self.n, self.n_pad = int(cap), n, n_pad_of(cap)
        self.device = torch.device(device)
        z = lambda c: torch.zeros(c, self.n_pad, device=self.device, dtype=torch.float32)
        self.raw = {k: z(c) for k, c in ROWS.items()}
        self.exp_avg = {k: z(c) for k, c in ROWS.items()}
        self.exp_avg_sq = {k: z(c) for k, c in ROWS.items()}
        self.grads = {k: z(c) for k, c in STORE_ROWS.items()}
        f = lambda x: torch.as_tensor(x, device=self.device, dtype=torch.float32).reshape(-1, n)
        # the inverse activations are the initial raw values (plain set-up, once)
        self.raw["means"][:, :n] = f(means)
        self.raw["log_scales"][:, :n] = torch.log(f(scales))
        self.raw["quats"][:, :n] = f(quats)
        o = f(opacity).clamp(1e-6, 1 - 1e-6)
        self.raw["logit_opacity"][:, :n] = torch.log(o / (1 - o))
        self.raw["rgb"][:, :n] = f(rgb)
        self.storage = {k: torch.zeros(c, self.n_pad, device=self.device, dtype=storage)
                        for k, c in STORE_ROWS.items()}
        self.storage["means"][:, :n] = f(means).to(storage)
        self.storage["scales"][:, :n] = f(scales).to(storage)
        self.storage["quats"][:, :n] = f(quats).to(storage)
        self.storage["opacity"][:, :n] = f(opacity).to(storage)
        self.storage["rgb"][:, :n] = f(rgb).to(storage)
        self.adam = adam if adam is not None else L.default_adam_opts(seed=seed)
        self.mcmc = mcmc if mcmc is not None else L.default_mcmc_opts(seed=seed)
        self.t = 0
        self.relocations = 0
        self._P = L.make_params(*(self.raw[k] for k in ROWS))
        self._M = L.make_params(*(self.exp_avg[k] for k in ROWS))
        self._V = L.make_params(*(self.exp_avg_sq[k] for k in ROWS))
        self._G = L.ss_splat_grads()
        self._G.means, self._G.scales, self._G.quats, self._G.opacity, self._G.rgb = (
            L.ptr(self.grads[k]) for k in STORE_ROWS)
        self._G.n_pad = self.n_pad
        self._ws = torch.empty(L.mcmc_workspace_size(self.cap), dtype=torch.uint8, device=self.device)

    @property
    def splats(self) -> L.ss_splats:
        """The rasterizer's view of the active splats."""
        s = self.storage
        return L.make_splats(s["means"], s["scales"], s["quats"], s["opacity"], s["rgb"], self.n)

    def zero_grad(self):
        for g in self.grads.values():
            g.zero_()

    def step(self, stream=None):
        """One fused Adam step (with the position noise) from ``self.grads``."""
        self.t += 1
        self.adam.step = self.t
        L.adam_step(self._P, self._M, self._V, self._G, self.splats, self.adam, stream)

    def relocate(self, stream=None) -> int:
        """3DGS-MCMC relocation of the dead splats and growth toward the budget; returns the new
        active count (synchronises the stream)."""
        self.mcmc.step = self.relocations
        self.relocations += 1
        self.n = L.mcmc_relocate(self._P, self._M, self._V, self.splats, self.cap, self.mcmc, self._ws, None,
                                 stream)
        return self.n
