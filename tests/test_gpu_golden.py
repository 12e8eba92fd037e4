"""The CUDA path, through the C ABI, against the golden fixtures of tests/golden: values that
follow from the paper's equations by hand (closed_forms.json) and the oracle's stored planes and
gradients of a small seeded scene with a camera delta, a colour correction, the sun view and the
distortion plane (oracle_scene.json).  Every pixel of both fixtures keeps a margin from the
threshold decisions, so all of them are compared."""
import numpy as np
import pytest
import torch

from paper_2606_28581_gb300 import _lib as L
from paper_2606_28581_gb300.frame import Frame, zero_grads
from tests.gpu_util import FWD_TOL, DeviceScene, grad_close, to_np
from tests.golden import fixtures as FX

pytestmark = pytest.mark.gpu

CLOSED = FX.load("closed_forms.json")
SCENE = FX.load("oracle_scene.json")


def _planes(out, i, sun, distortion=False):
    p = dict(depth=to_np(out.depth[i]), alpha=to_np(out.alpha[i]), T=to_np(out.T_final[i]))
    if not sun:
        p.update(rgb=to_np(out.rgb[i]), normal=to_np(out.normal[i]))
        if distortion:
            p["distort"] = to_np(out.distort[i])
    return p


@pytest.mark.parametrize("name", [c["name"] for c in CLOSED["cases"]])
def test_closed_forms(name):
    case = next(c for c in CLOSED["cases"] if c["name"] == name)
    sun = case["view"] == "sun"
    ds = DeviceScene(FX.scene_of(case))
    frame = Frame(ds.scene.cameras, L.SS_PASS_SUN if sun else L.SS_PASS_MAIN)
    out = frame.forward(ds.splats, ds.dF, ds.color)
    torch.cuda.synchronize()
    planes = _planes(out, 0, sun)
    for key, want in case["expected"].items():
        got = np.array([planes[key][..., j, i] for (i, j) in case["pixels"]])
        err = np.abs(got - np.asarray(want)).max()
        assert err <= FWD_TOL, (key, got, want)
    for (i, j), a in zip(case["pixels"], case["expected"].get("alpha", [])):
        if a == 0.0:
            assert planes["alpha"][j, i] == 0.0
    if "grad" not in case:
        return
    g = case["grad"]
    i, j = g["pixel"]
    cam = ds.scene.cameras[0]
    ups = dict(alpha=torch.zeros(cam.height, cam.width, device="cuda"),
               rgb=torch.zeros(3, cam.height, cam.width, device="cuda"))
    ups["alpha"][j, i] = g["d_alpha"]
    ups["rgb"][:, j, i] = torch.tensor(g["d_rgb"], device="cuda")
    grads = zero_grads(ds.n_pad, "cuda")
    frame.backward(ds.splats, out, [ups], grads)
    torch.cuda.synchronize()
    for key, want in g["expected"].items():
        got = grads[key][:, :ds.n].cpu().numpy().astype(np.float64).reshape(-1)
        grad_close(got, np.asarray(want), name=key)


def test_stored_scene_forward_and_backward():
    sc = FX.scene_of(SCENE)
    ds = DeviceScene(sc)
    frame = Frame(sc.cameras, L.SS_PASS_MAIN | L.SS_PASS_SUN, distortion=True)
    out = frame.forward(ds.splats, ds.dF, ds.color)
    torch.cuda.synchronize()
    ups = []
    for i, t in enumerate(frame.targets):
        want = SCENE["sun" if t.sun else "main"]
        planes = _planes(out, i, t.sun, distortion=True)
        for key, w in want.items():
            err = np.abs(planes[key] - np.asarray(w)).max()
            assert err <= FWD_TOL, (t.sun, key, err)
        u = FX.upstream(t.width, t.height, t.sun)
        ups.append({k: torch.from_numpy(v.astype(np.float32)).cuda() for k, v in u.items()})
    grads = zero_grads(ds.n_pad, "cuda")
    d_dF = torch.zeros(1, 2, 4, device="cuda")
    d_col = torch.zeros(1, 3, 4, device="cuda")
    frame.backward(ds.splats, out, ups, grads, d_dF=d_dF, d_color=d_col)
    torch.cuda.synchronize()
    gm, gs = SCENE["grad_main"], SCENE["grad_sun"]
    for key in ("means", "scales", "quats", "opacity", "rgb"):
        got = grads[key][:, :ds.n].cpu().numpy().astype(np.float64)
        want = np.asarray(gm[key]).reshape(got.shape) + np.asarray(gs[key]).reshape(got.shape)
        grad_close(got, want, name=key)
    grad_close(to_np(d_dF[0]), np.asarray(gm["dF"]) + np.asarray(gs["dF"]), name="dF")
    grad_close(to_np(d_col[0]), np.asarray(gm["color"]), name="color")
