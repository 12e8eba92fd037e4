"""Sun visibility and image formation (K7) against the FP64 shading oracle, through the C ABI.

The FP64 oracle renders a view and its sun view; the planes, rounded to float32, are the input
of both the shading kernels and the shading oracle (widened back exactly), so the comparison
isolates the shading arithmetic.  Pixels whose decisions sit within FP32 reach of a threshold
are excluded (and counted).  The chain test at the end runs the whole path on the GPU."""
import numpy as np
import pytest
import torch

import scenegen
from oracle import shade as S
from paper_2606_28581_gb300 import _lib as L
from paper_2606_28581_gb300.frame import Frame
from tests.gpu_util import grad_close, to_np
from tests.tolerances import CHAIN_GRAD_FLOOR

pytestmark = pytest.mark.gpu

K, EPS = 60.0, 1e-3


def _scene(seed):
    return scenegen.make_scene(n=6000, extent_m=80.0, seed=seed, views=[
        dict(width=120, height=90, off_nadir=20.0, delta=True, color_noise=0.02),
        dict(width=96, height=80, off_nadir=12.0, delta=True, color_noise=0.02)])


def _planes(scene):
    """Each view's planes and its sun view's, rendered by the FP64 oracle and rounded to float32
    (on the device), and the cameras' deltas."""
    import oracle
    s64 = oracle.SceneF64.of(scene)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    planes = []
    for cam in scene.cameras:
        om = oracle.render(s64, cam, color=cam.color)
        osun = oracle.render(s64, cam, sun=True)
        planes.append(dict(rgb=f(om["rgb"]), depth=f(om["depth"]), alpha=f(om["alpha"]), sun_depth=f(osun["depth"]),
                           sun_alpha=f(osun["alpha"])))
    dF = torch.from_numpy(np.stack([c.dF_xy for c in scene.cameras]).astype(np.float32)).cuda()
    return planes, dF


def _views(planes, extra):
    return [dict(planes[c], **extra[c]) for c in range(len(planes))]


def _margin_keep(scene, planes, c, k, bias):
    m, frac = S.shade_margin(planes["depth"], planes["alpha"], planes["sun_depth"], planes["sun_alpha"],
                             scene.cameras[c], k, bias, EPS)
    return m > 1e-3


@pytest.mark.parametrize("bias", [0.0, 0.01])
def test_shade_forward_matches_oracle(bias):
    scene = _scene(seed=21)
    planes, dF = _planes(scene)
    V = len(scene.cameras)
    La = torch.tensor([[0.2, 0.3, 0.4], [0.5, 0.35, 0.25]], device="cuda")
    imgs = [torch.empty(3, c.height, c.width, device="cuda") for c in scene.cameras]
    vis = [torch.empty(c.height, c.width, device="cuda") for c in scene.cameras]
    views = _views(planes, [dict(image=imgs[c], vis=vis[c]) for c in range(V)])
    cams = L.make_cameras(scene.cameras)
    opts = L.default_shade_opts(esm_k=K, esm_bias=bias, alpha_eps=EPS)
    L.shade_fwd(cams, V, dF, La, opts, L.shade_io_array(views))
    torch.cuda.synchronize()
    shadowed = 0
    for c in range(V):
        p = {k: to_np(views[c][k]) for k in ("rgb", "depth", "alpha", "sun_depth", "sun_alpha")}
        I, Vo = S.shade_forward(p["rgb"], p["depth"], p["alpha"], p["sun_depth"], p["sun_alpha"], scene.cameras[c],
                                to_np(La[c]), K, bias, EPS, dF=to_np(dF[c]))
        keep = _margin_keep(scene, p, c, K, bias)
        assert keep.mean() > 0.98
        assert np.abs(to_np(vis[c]) - Vo)[keep].max() <= 1e-5
        assert np.abs(to_np(imgs[c]) - I)[:, keep].max() <= 1e-5
        shadowed += int((Vo[keep] < 0.99).sum())
    assert shadowed > 100  # the scene casts shadows


def test_shade_backward_matches_oracle():
    scene = _scene(seed=22)
    planes, dF = _planes(scene)
    V = len(scene.cameras)
    rng = np.random.default_rng(3)
    La = torch.tensor([[0.3, 0.2, 0.4], [0.45, 0.5, 0.3]], device="cuda")
    zeros = lambda t: torch.zeros_like(t)
    d_img, extra, keeps = [], [], []
    for c in range(V):
        cam = scene.cameras[c]
        p = {k: to_np(planes[c][k]) for k in ("depth", "alpha", "sun_depth", "sun_alpha")}
        keep = _margin_keep(scene, p, c, K, 0.0)
        keeps.append(keep)
        dI = rng.normal(size=(3, cam.height, cam.width)) * keep
        d_img.append(torch.from_numpy(dI.astype(np.float32)).cuda())
        extra.append(dict(image=torch.empty(3, cam.height, cam.width, device="cuda"), d_image=d_img[c],
                          d_rgb=zeros(planes[c]["rgb"]), d_depth=zeros(planes[c]["depth"]),
                          d_alpha=zeros(planes[c]["alpha"]), d_sun_depth=zeros(planes[c]["sun_depth"]),
                          d_sun_alpha=zeros(planes[c]["sun_alpha"])))
    views = _views(planes, extra)
    cams = L.make_cameras(scene.cameras)
    opts = L.default_shade_opts(esm_k=K, esm_bias=0.0, alpha_eps=EPS)
    d_La = torch.zeros(V, 3, device="cuda")
    d_dF = torch.zeros(V, 2, 4, device="cuda")
    L.shade_bwd(cams, V, dF, La, opts, L.shade_io_array(views), d_La, d_dF)
    torch.cuda.synchronize()
    for c in range(V):
        v = views[c]
        p = {k: to_np(v[k]) for k in ("rgb", "depth", "alpha", "sun_depth", "sun_alpha")}
        g = S.shade_backward(to_np(d_img[c]), p["rgb"], p["depth"], p["alpha"], p["sun_depth"], p["sun_alpha"],
                             scene.cameras[c], to_np(La[c]), K, 0.0, EPS, dF=to_np(dF[c]))
        for key in ("rgb", "depth", "alpha", "sun_depth", "sun_alpha"):
            grad_close(to_np(v["d_" + key]), g[key], name=f"view {c} d_{key}")
        grad_close(to_np(d_La[c]), g["La"], name=f"view {c} d_La")
        grad_close(to_np(d_dF[c]), g["dF"], name=f"view {c} d_dF")
    assert any(np.abs(to_np(views[c]["d_sun_depth"])).max() > 0 for c in range(V))  # shadows carry gradient


def test_shade_rejects_bad_arguments():
    scene = _scene(seed=23)
    cams = L.make_cameras(scene.cameras)
    La = torch.zeros(2, 3, device="cuda")
    opts = L.default_shade_opts()
    io = L.shade_io_array([{}, {}])  # no planes
    assert L.load().ss_shade_fwd(cams, 2, None, L.ptr(La), opts, io, None) == L.SS_ERR_INVALID_ARG
    bad = L.default_shade_opts(alpha_eps=0.0)
    assert L.load().ss_shade_fwd(cams, 2, None, L.ptr(La), bad, io, None) == L.SS_ERR_INVALID_ARG


def test_render_and_shade_chain_matches_oracle_chain():
    """The differentiable chain render -> shade -> loss on the GPU (autograd forms) against the
    FP64 chain: oracle render of each view and its sun view, oracle shading and its adjoint, and
    the oracle rasterizer adjoint of the upstream planes that the shading adjoint leaves.  Main
    pixels near a decision of either stage, or sampling a sun texel near one, carry no weight."""
    import oracle
    from paper_2606_28581_gb300.autograd import render, shade
    from tests.gpu_util import MARGIN

    scene = scenegen.make_scene(n=3000, extent_m=60.0, seed=24, views=[
        dict(width=80, height=64, off_nadir=18.0, delta=True, color_noise=0.02)])
    cam = scene.cameras[0]
    t = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda", requires_grad=True)
    P = dict(means=t(scene.means), scales=t(scene.scales), quats=t(scene.quats), opacity=t(scene.opacity),
             rgb=t(scene.rgb), dF=t(np.stack([c.dF_xy for c in scene.cameras])),
             color=t(np.stack([c.color for c in scene.cameras])))
    La = torch.tensor([[0.3, 0.35, 0.4]], device="cuda", requires_grad=True)
    opts = L.default_shade_opts(esm_k=K, esm_bias=0.0, alpha_eps=EPS)
    # FP64 chain
    s64 = oracle.SceneF64.of(scene)
    om = oracle.render(s64, cam, sun=False, color=cam.color)
    os_ = oracle.render(s64, cam, sun=True)
    planes = dict(rgb=om["rgb"], depth=om["depth"], alpha=om["alpha"], sun_depth=os_["depth"], sun_alpha=os_["alpha"])
    keep = _margin_keep(scene, planes, 0, K, 0.0) & (om["margin_bwd"] >= MARGIN)
    g = S._geometry(planes["depth"], planes["alpha"], planes["sun_depth"], planes["sun_alpha"], cam, None, EPS)
    sun_ok = os_["margin_bwd"] >= MARGIN
    for di, dj in g["taps"]:
        keep &= sun_ok[g["jc"] + dj, g["ic"] + di]
    assert keep.mean() > 0.95
    wI = np.random.default_rng(9).normal(size=(3, cam.height, cam.width)) * keep
    La64 = np.array([0.3, 0.35, 0.4])
    gs = S.shade_backward(wI, planes["rgb"], planes["depth"], planes["alpha"], planes["sun_depth"],
                          planes["sun_alpha"], cam, La64, K, 0.0, EPS)
    gm = oracle.backward(s64, cam, dict(rgb=gs["rgb"], depth=gs["depth"], alpha=gs["alpha"]), color=cam.color)
    gsun = oracle.backward(s64, cam, dict(depth=gs["sun_depth"], alpha=gs["sun_alpha"]), sun=True)
    # GPU chain
    frame = Frame(scene.cameras, L.SS_PASS_MAIN | L.SS_PASS_SUN)
    outs = render(frame, P["means"], P["scales"], P["quats"], P["opacity"], P["rgb"], P["dF"], P["color"])
    img = shade(frame, outs, La, P["dF"], opts)
    loss = (img[0]["image"] * torch.from_numpy(wI.astype(np.float32)).cuda()).sum()
    loss.backward()
    # the GPU chain shades the FP32 rasterizer outputs, and the sun-visibility test amplifies their
    # errors: FP32-sized plane errors alone move the FP64 chain's gradients beyond the default
    # per-element floor (tests/test_fp32_bounds.py); the per-tensor bound stays 1e-3
    for k in ("means", "scales", "quats", "opacity", "rgb"):
        grad_close(to_np(P[k].grad).reshape(-1), (gm[k] + gsun[k]).reshape(-1), name=k, floor=CHAIN_GRAD_FLOOR)
    grad_close(to_np(P["dF"].grad[0]), gm["dF"] + gsun["dF"] + gs["dF"], name="dF", floor=CHAIN_GRAD_FLOOR)
    grad_close(to_np(P["color"].grad[0]), gm["color"], name="color", floor=CHAIN_GRAD_FLOOR)
    grad_close(to_np(La.grad[0]), gs["La"], name="La", floor=CHAIN_GRAD_FLOOR)
