"""Depth-gradient surface normal (K8) against the FP64 oracle, through the C ABI and the autograd
form: on planes the FP64 oracle renders, rounded to float32 and given to both sides (isolating
the normal arithmetic), and end to end as the normal-consistency regulariser alpha - n . N
(render -> depth_normal chain on the GPU against the oracle chain)."""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from oracle import normals as NO
from paper_2606_28581_gb300 import _lib as L
from paper_2606_28581_gb300.frame import Frame
from tests.gpu_util import MARGIN, grad_close, to_np
from tests.tolerances import CHAIN_GRAD_FLOOR, NORMAL_FWD_TOL, NORMAL_GRAD_FLOOR

pytestmark = pytest.mark.gpu

EPS = 1e-3


def _scene(seed):
    return scenegen.make_scene(n=5000, extent_m=70.0, seed=seed, views=[
        dict(width=110, height=84, off_nadir=22.0, delta=True, color_noise=0.02),
        dict(width=90, height=70, off_nadir=8.0, delta=True)])


def _alpha_margin(alpha):
    """Pixels whose normal could be decided differently in FP32: its own or a neighbour's alpha
    within 1e-3 (relative) of eps."""
    near = np.abs(alpha - EPS) < 1e-3 * EPS
    bad = near.copy()
    bad[1:, :] |= near[:-1, :]
    bad[:-1, :] |= near[1:, :]
    bad[:, 1:] |= near[:, :-1]
    bad[:, :-1] |= near[:, 1:]
    return ~bad


def test_depth_normal_matches_oracle_forward_and_backward():
    scene = _scene(31)
    s64 = oracle.SceneF64.of(scene)
    dF = torch.from_numpy(np.stack([c.dF_xy for c in scene.cameras]).astype(np.float32)).cuda()
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    V = len(scene.cameras)
    cams = L.make_cameras(scene.cameras)
    rng = np.random.default_rng(4)
    views = []
    for c in range(V):
        cam = scene.cameras[c]
        om = oracle.render(s64, cam, color=cam.color)
        views.append(dict(depth=f(om["depth"]), alpha=f(om["alpha"]),
                          normal=torch.empty(3, cam.height, cam.width, device="cuda")))
    L.depth_normal_fwd(cams, V, dF, EPS, L.dnormal_io_array(views))
    torch.cuda.synchronize()
    dNs, keeps = [], []
    for c in range(V):
        cam = scene.cameras[c]
        d, a = to_np(views[c]["depth"]), to_np(views[c]["alpha"])
        N, ok = NO.depth_normal(d, a, cam, EPS, dF=to_np(dF[c]))
        keep = _alpha_margin(a)
        keeps.append(keep)
        assert ok.mean() > 0.5
        assert np.abs(to_np(views[c]["normal"]) - N)[:, keep].max() <= NORMAL_FWD_TOL
        dNs.append(rng.normal(size=(3, cam.height, cam.width)) * keep)
        views[c].update(d_normal=torch.from_numpy(dNs[c].astype(np.float32)).cuda(),
                        d_depth=torch.zeros_like(views[c]["depth"]), d_alpha=torch.zeros_like(views[c]["alpha"]))
    d_dF = torch.zeros(V, 2, 4, device="cuda")
    L.depth_normal_bwd(cams, V, dF, EPS, L.dnormal_io_array(views), d_dF)
    torch.cuda.synchronize()
    for c in range(V):
        d, a = to_np(views[c]["depth"]), to_np(views[c]["alpha"])
        g = NO.depth_normal_backward(dNs[c], d, a, scene.cameras[c], EPS, dF=to_np(dF[c]))
        grad_close(to_np(views[c]["d_depth"]), g["depth"], name=f"view {c} d_depth")
        grad_close(to_np(views[c]["d_alpha"]), g["alpha"], name=f"view {c} d_alpha")
        grad_close(to_np(d_dF[c]), g["dF"], name=f"view {c} d_dF")


def test_normal_consistency_chain_matches_oracle_chain():
    """L = sum w (alpha - n_rendered . N): render -> depth_normal on the GPU against the FP64 chain
    (oracle render, oracle normal and its adjoint, oracle rasterizer adjoint).  A pixel carries
    no weight when it or a neighbour is near a rasterizer decision."""
    from paper_2606_28581_gb300.autograd import depth_normal, render

    scene = scenegen.make_scene(n=2500, extent_m=50.0, seed=32, views=[
        dict(width=72, height=60, off_nadir=16.0, delta=True, color_noise=0.02)])
    cam = scene.cameras[0]
    t = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda", requires_grad=True)
    P = dict(means=t(scene.means), scales=t(scene.scales), quats=t(scene.quats), opacity=t(scene.opacity),
             rgb=t(scene.rgb), dF=t(np.stack([c.dF_xy for c in scene.cameras])),
             color=t(np.stack([c.color for c in scene.cameras])))
    s64 = oracle.SceneF64.of(scene)
    om = oracle.render(s64, cam, color=cam.color)
    good = om["margin_bwd"] >= MARGIN
    keep = good.copy()
    keep[1:, :] &= good[:-1, :]
    keep[:-1, :] &= good[1:, :]
    keep[:, 1:] &= good[:, :-1]
    keep[:, :-1] &= good[:, 1:]
    keep &= _alpha_margin(om["alpha"])
    assert keep.mean() > 0.9
    w = np.random.default_rng(8).normal(size=(cam.height, cam.width)) * keep
    # FP64 chain: dL/dalpha = w (+ through N), dL/dn = -w N, dL/dN = -w n
    N, _ = NO.depth_normal(om["depth"], om["alpha"], cam, EPS)
    gN = NO.depth_normal_backward(-w[None] * om["normal"], om["depth"], om["alpha"], cam, EPS)
    up = dict(alpha=w + gN["alpha"], depth=gN["depth"], normal=-w[None] * N)
    ref = oracle.backward(s64, cam, up, color=cam.color)
    # GPU chain
    frame = Frame(scene.cameras, L.SS_PASS_MAIN)
    outs = render(frame, P["means"], P["scales"], P["quats"], P["opacity"], P["rgb"], P["dF"], P["color"])
    Ng = depth_normal(frame, outs, P["dF"], EPS)
    W_ = torch.from_numpy(w.astype(np.float32)).cuda()
    loss = (W_ * (outs[0]["alpha"] - (outs[0]["normal"] * Ng[0]).sum(0))).sum()
    loss.backward()
    # the GPU chain works on FP32 rasterized planes; the FP32-sized plane errors alone move the FP64
    # chain's gradients beyond the default per-element floor (tests/test_fp32_bounds.py)
    for k in ("means", "scales", "quats", "opacity", "rgb"):
        grad_close(to_np(P[k].grad).reshape(-1), ref[k].reshape(-1), name=k, floor=CHAIN_GRAD_FLOOR)
    grad_close(to_np(P["dF"].grad[0]), ref["dF"] + gN["dF"], name="dF", floor=CHAIN_GRAD_FLOOR)


def test_depth_normal_full_size_views():
    """Three large ragged views (several 32 x 32 tiles per block in both kernels' tile loops) on
    host-generated planes: a smooth height field with holes (alpha = 0) and alpha in [0.05, 1];
    every pixel against the oracle."""
    scene = scenegen.make_scene(n=64, extent_m=400.0, seed=33, views=[
        dict(width=1500, height=1300, off_nadir=18.0, delta=True),
        dict(width=1100, height=2000, off_nadir=9.0, delta=True),
        dict(width=2048, height=1024, off_nadir=27.0, delta=False)])
    V = len(scene.cameras)
    cams = L.make_cameras(scene.cameras)
    dF = torch.from_numpy(np.stack([c.dF_xy for c in scene.cameras]).astype(np.float32)).cuda()
    rng = np.random.default_rng(34)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    views, planes = [], []
    for cam in scene.cameras:
        y, x = np.mgrid[0:cam.height, 0:cam.width].astype(np.float64)
        z = 1.0 + 0.2 * np.sin(x / 37.0) * np.cos(y / 53.0) + 0.05 * np.sin((x + 2 * y) / 11.0)
        a = rng.uniform(0.05, 1.0, z.shape)
        a[rng.uniform(size=z.shape) < 0.02] = 0.0  # holes: no surface
        a32 = a.astype(np.float32)
        d32 = (a32.astype(np.float64) * z).astype(np.float32)
        planes.append((d32.astype(np.float64), a32.astype(np.float64)))
        views.append(dict(depth=f(d32), alpha=f(a32), normal=torch.empty(3, cam.height, cam.width, device="cuda")))
    L.depth_normal_fwd(cams, V, dF, EPS, L.dnormal_io_array(views))
    torch.cuda.synchronize()
    dNs = []
    for c, cam in enumerate(scene.cameras):
        d, a = planes[c]
        N, ok = NO.depth_normal(d, a, cam, EPS, dF=to_np(dF[c]))
        assert ok.mean() > 0.8
        assert np.abs(to_np(views[c]["normal"]) - N).max() <= NORMAL_FWD_TOL
        dN = rng.normal(size=(3, cam.height, cam.width))
        dNs.append(dN.astype(np.float32).astype(np.float64))
        views[c].update(d_normal=f(dNs[c]), d_depth=torch.zeros_like(views[c]["depth"]),
                        d_alpha=torch.zeros_like(views[c]["alpha"]))
    d_dF = torch.zeros(V, 2, 4, device="cuda")
    L.depth_normal_bwd(cams, V, dF, EPS, L.dnormal_io_array(views), d_dF)
    torch.cuda.synchronize()
    for c, cam in enumerate(scene.cameras):
        d, a = planes[c]
        g = NO.depth_normal_backward(dNs[c], d, a, cam, EPS, dF=to_np(dF[c]))
        # a pixel's depth gradient sums its four neighbours' contributions, which reach ~2e4 here
        # and can cancel to ~1; one FP32 rounding of z = D / alpha already moves such pixels beyond
        # the default per-element floor (tests/test_fp32_bounds.py); the global bound stays 1e-3
        grad_close(to_np(views[c]["d_depth"]), g["depth"], name=f"view {c} d_depth", floor=NORMAL_GRAD_FLOOR)
        grad_close(to_np(views[c]["d_alpha"]), g["alpha"], name=f"view {c} d_alpha", floor=NORMAL_GRAD_FLOOR)
        grad_close(to_np(d_dF[c]), g["dF"], name=f"view {c} d_dF")
