"""Parity at the full workload sizes, in the launch configuration the bench times: the batched
persistent step replayed from its CUDA graphs (1M splats, 16 views of uneven size, BF16 storage),
the single 2048^2 view with its shadow pass (FP32 and BF16 storage), and the 4M-splat, 32-view
step.  The oracle renders seeded crops of a few targets one by one; the backward runs with
upstream gradients that are zero outside those crops, so the GPU's whole-frame gradients must
equal the oracle's crop gradients."""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from paper_2606_28581_gb300 import _lib as L
from paper_2606_28581_gb300.batched import BatchedStep
from paper_2606_28581_gb300.frame import Frame
from tests.gpu_util import (BF16_TOL, FWD_TOL, MARGIN, MAX_EXCLUDED, DeviceScene, check_forward, grad_close,
                            to_np)

pytestmark = pytest.mark.gpu

CROP = 96  # crops never overlap: each picked target gets one


def _crops(frame, picks, seed):
    """(target index, crop) for the picked targets, crops seeded inside each target."""
    rng = np.random.default_rng(seed)
    out = []
    for ti in picks:
        t = frame.targets[ti]
        w, h = min(CROP, t.width), min(CROP, t.height)
        out.append((ti, (int(rng.integers(0, t.width - w + 1)), int(rng.integers(0, t.height - h + 1)), w, h)))
    return out


def _zero_upstream(frame, distortion=False):
    ups = []
    for t in frame.targets:
        z = lambda c: torch.zeros((c, t.height, t.width) if c > 1 else (t.height, t.width), device="cuda")
        u = dict(depth=z(1), alpha=z(1))
        if not t.sun:
            u.update(rgb=z(3), normal=z(3))
            if distortion:
                u["distort"] = z(1)
        ups.append(u)
    return ups


def _check_step(scene, ds, frame, out, run_backward, upstream, crops, tol, seed, distortion=False):
    """Forward planes of every crop against the oracle; then the backward with upstream
    gradients inside the crops (margin pixels zeroed) against the oracle's crop adjoint.  With
    ``distortion`` the main targets' distortion planes and their upstream are included."""
    s64 = ds.stored_scene64()
    rng = np.random.default_rng(seed)
    V = len(scene.cameras)
    ref = None
    excluded = []  # margin pixels are bounded over all crops together: one small crop is a noisy sample
    for ti, crop in crops:
        t = frame.targets[ti]
        cam = scene.cameras[t.cam]
        ora = oracle.render(s64, cam, sun=t.sun, crop=crop, color=None if t.sun else cam.color)
        gpu = dict(depth=to_np(out.depth[ti]), alpha=to_np(out.alpha[ti]))
        if not t.sun:
            gpu.update(rgb=to_np(out.rgb[ti]), normal=to_np(out.normal[ti]))
        _, exc = check_forward(gpu, ora, sun=t.sun, tol=tol, crop=crop, max_excluded=None)
        excluded.append(exc)
        if distortion and not t.sun:
            x0, y0, w, h = crop
            dd = np.abs(to_np(out.distort[ti])[y0:y0 + h, x0:x0 + w] - ora["distort"])
            assert dd[ora["margin_fwd"] >= MARGIN].max() <= tol, dd.max()
        # upstream inside the crop, zero on margin pixels
        x0, y0, w, h = crop
        keep = (ora["margin_bwd"] >= MARGIN).astype(np.float64)
        r, d, n, a = scenegen.upstream_grads(rng, h, w, sun=t.sun)
        u_np = dict(depth=d * keep, alpha=a * keep)
        if not t.sun:
            u_np.update(rgb=r * keep, normal=n * keep)
            if distortion:
                u_np["distort"] = rng.normal(size=(h, w)) * keep
        for k, v in u_np.items():
            upstream[ti][k][..., y0:y0 + h, x0:x0 + w] = torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda()
        u64 = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in u_np.items()}
        g = oracle.backward(s64, cam, u64, sun=t.sun, crop=crop, color=None if t.sun else cam.color)
        g["dF_v"] = np.zeros((V, 2, 4))
        g["dF_v"][t.cam] = g["dF"]
        g["color_v"] = np.zeros((V, 3, 4))
        if not t.sun:
            g["color_v"][t.cam] = g["color"]
        ref = g if ref is None else {k: ref[k] + g[k] for k in ref}
    assert float(np.mean(excluded)) <= MAX_EXCLUDED, f"too many margin pixels: {excluded}"
    grads, d_dF, d_color = run_backward()
    n = ds.n
    for k in ("means", "scales", "quats", "opacity", "rgb"):
        gg = grads[k][:, :n].cpu().numpy().astype(np.float64)
        grad_close(gg, ref[k].reshape(gg.shape), name=k)
    grad_close(d_dF.cpu().numpy().astype(np.float64), ref["dF_v"], name="dF")
    grad_close(d_color.cpu().numpy().astype(np.float64), ref["color_v"], name="color")


def _batched_parity(name, picks, seed, distortion=False):
    scene = scenegen.workload(name)
    ds = DeviceScene(scene, dtype=torch.bfloat16)
    probe = Frame(scene.cameras, L.SS_PASS_MAIN | L.SS_PASS_SUN)
    ups = _zero_upstream(probe, distortion)
    splats = dict(means=ds.means, scales=ds.scales, quats=ds.quats, opacity=ds.opacity, rgb=ds.rgb)
    step = BatchedStep(scene.cameras, splats, ds.n, ds.dF, ds.color, ups, opts=L.default_opts(persistent=1),
                       distortion=distortion)
    step.capture()
    step.replay()
    torch.cuda.synchronize()
    st, needed, walked, flags = step.check()
    assert st == L.SS_OK and flags == 0
    crops = _crops(step.frame, picks(len(scene.cameras)), seed)

    def run_backward():
        step.replay()
        torch.cuda.synchronize()
        return step.grads, step.d_dF, step.d_color

    _check_step(scene, ds, step.frame, step.out, run_backward, ups, crops, BF16_TOL, seed, distortion)


def test_batched_1M_16_views_bf16_graph_step():
    """1M splats, 16 views of uneven size with camera deltas, their shadow passes, BF16 storage,
    persistent launches replayed from the CUDA graphs: crops of three views and two sun views."""
    _batched_parity("batched", lambda V: [0, V // 2, V - 1, V + 1, 2 * V - 2], seed=31)


def test_batched_1M_16_views_bf16_graph_step_with_distortion():
    """The same step with the distortion plane written by the forward and back-propagated from
    the crops (the launch configuration of the bench's distortion line)."""
    _batched_parity("batched", lambda V: [1, V // 2 + 1, V + 3], seed=35, distortion=True)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_single_2048_view_with_shadow_pass(dtype):
    """500k splats, one 2048^2 view with colour correction and its 1024^2 shadow pass, plain
    single-view path (FP32 storage) and BF16 storage."""
    scene = scenegen.workload("single")
    ds = DeviceScene(scene, dtype=dtype)
    frame = Frame(scene.cameras, L.SS_PASS_MAIN | L.SS_PASS_SUN)
    out = frame.forward(ds.splats, ds.dF, ds.color)
    torch.cuda.synchronize()
    ups = _zero_upstream(frame)
    crops = _crops(frame, [0, 1], seed=32)

    def run_backward():
        grads = {k: torch.zeros(c, ds.n_pad, device="cuda") for k, c in
                 (("means", 3), ("scales", 2), ("quats", 4), ("opacity", 1), ("rgb", 3))}
        d_dF = torch.zeros(1, 2, 4, device="cuda")
        d_col = torch.zeros(1, 3, 4, device="cuda")
        frame.backward(ds.splats, out, ups, grads, d_dF=d_dF, d_color=d_col)
        torch.cuda.synchronize()
        return grads, d_dF, d_col

    tol = FWD_TOL if dtype == torch.float32 else BF16_TOL
    _check_step(scene, ds, frame, out, run_backward, ups, crops, tol, seed=33)


def test_full_4M_32_views_bf16_graph_step():
    """4M splats over 2 x 2 km, 32 views at 2048^2 with deltas, colour correction and shadow
    passes, BF16 storage, graph-replayed persistent step: crops of two views and a sun view."""
    _batched_parity("full", lambda V: [3, V - 5, V + 9], seed=34)
