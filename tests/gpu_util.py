"""Shared helpers of the GPU tests: move seeded scenes to the device, run the CUDA path
through the C ABI, and compare with the oracle under the decision-margin exclusion."""
import numpy as np
import torch

import oracle
import scenegen
from paper_2606_28581_gb300 import _lib as L
from paper_2606_28581_gb300.frame import Frame, n_pad_of, pad_planar

DEV = "cuda"
FWD_TOL = 1e-5        # absolute, FP32 storage (all outputs)
BF16_TOL = 2e-3       # absolute, BF16 storage (against the oracle on the stored values)
GRAD_TOL = 1e-3       # relative (see grad_close)
MARGIN = 2e-5         # pixels whose closest threshold decision is nearer than this are excluded
MAX_EXCLUDED = 1e-3   # fraction of pixels that may be excluded


class DeviceScene:
    def __init__(self, scene, dtype=torch.float32):
        self.scene = scene
        self.dtype = dtype
        n = scene.n
        self.n = n
        self.n_pad = n_pad_of(n)
        t = lambda a: pad_planar(torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(DEV).to(dtype),
                                 self.n_pad)
        self.means, self.scales, self.quats = t(scene.means), t(scene.scales), t(scene.quats)
        self.opacity, self.rgb = t(scene.opacity[None]), t(scene.rgb)
        self.splats = L.make_splats(self.means, self.scales, self.quats, self.opacity, self.rgb, n)
        self.dF = torch.from_numpy(np.stack([c.dF_xy for c in scene.cameras]).astype(np.float32)).to(DEV)
        self.color = torch.from_numpy(np.stack([c.color for c in scene.cameras]).astype(np.float32)).to(DEV)

    def stored_scene64(self):
        """The stored values (after any BF16 rounding, done here on the host), widened exactly,
        for the oracle."""
        sc = self.scene
        r = (lambda a: scenegen.to_bf16_exact(np.asarray(a, np.float32))) if self.dtype == torch.bfloat16 else \
            (lambda a: np.asarray(a, np.float32))
        g = lambda a: r(a).astype(np.float64)
        return oracle.SceneF64(g(sc.means), g(sc.scales), g(sc.quats), g(sc.opacity), g(sc.rgb))


def run_forward(ds: DeviceScene, passes=L.SS_PASS_MAIN, opts=None, cams=None):
    frame = Frame(cams if cams is not None else ds.scene.cameras, passes, opts)
    out = frame.forward(ds.splats, ds.dF, ds.color)
    torch.cuda.synchronize()
    return frame, out


def to_np(x):
    return None if x is None else x.detach().float().cpu().numpy().astype(np.float64)


def oracle_forward(s64, cam, sun=False, crop=None):
    return oracle.render(s64, cam, sun=sun, crop=crop, color=None if sun else cam.color)


def check_forward(gpu: dict, ora: dict, sun: bool, tol: float, margin: float = MARGIN, crop=None,
                  max_excluded=MAX_EXCLUDED):
    """Element-wise comparison on all pixels whose decision margin is >= margin.  The fraction of
    excluded pixels is asserted here unless ``max_excluded`` is None (the caller then bounds the
    total over several crops)."""
    keep = ora["margin_fwd"] >= margin
    excluded = 1.0 - keep.mean()
    if max_excluded is not None:
        assert excluded <= max_excluded, f"too many margin pixels: {excluded:.4%}"
    sl = (slice(None),) if crop is None else (slice(crop[1], crop[1] + crop[3]), slice(crop[0], crop[0] + crop[2]))
    names = ["depth", "alpha"] + ([] if sun else ["rgb", "normal"])
    errs = {}
    for k in names:
        g = gpu[k]
        g = g[..., sl[0], sl[1]] if crop is not None else g
        d = np.abs(g - ora[k])
        d = d[..., keep] if d.ndim == 3 else d[keep]
        errs[k] = float(d.max()) if d.size else 0.0
    for k, e in errs.items():
        assert e <= tol, f"{k}: max abs err {e:.3e} > {tol:.1e} (all errors {errs})"
    return errs, excluded


def grad_close(g: np.ndarray, ref: np.ndarray, rtol=GRAD_TOL, name="", floor=1e-3):
    """max|g - ref| <= rtol max|ref| and per element |g - ref| <= rtol (|ref| + floor max|ref|)."""
    scale = float(np.abs(ref).max())
    if scale == 0.0:
        assert float(np.abs(g).max()) == 0.0, name
        return 0.0
    d = np.abs(g - ref)
    assert d.max() <= rtol * scale, f"{name}: max err {d.max():.3e} vs {rtol * scale:.3e}"
    bound = rtol * (np.abs(ref) + floor * scale)
    bad = d > bound
    if bad.any():
        i = int(np.argmax(np.where(bad, d / bound, 0.0)))
        raise AssertionError(f"{name}: {bad.sum()} elements outside the per-element bound; worst at {i}: "
                             f"got {g.flat[i]:.6e}, oracle {ref.flat[i]:.6e}, bound {bound.flat[i]:.3e}, "
                             f"largest |oracle| {scale:.3e}")
    return float(d.max() / scale)
