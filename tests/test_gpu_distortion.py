"""Distortion of the blending weights (the point-sample distortion that the training loss of
Supp. B adds) on the CUDA path against the FP64 oracle, through the C ABI, the batched graph
step and the autograd form."""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from paper_2606_28581_gb300 import _lib as L
from paper_2606_28581_gb300.frame import Frame, grads_struct, zero_grads
from tests.gpu_util import FWD_TOL, MARGIN, DeviceScene, check_forward, grad_close, oracle_forward, to_np
from tests.test_gpu_parity import SCENES, gpu_planes, ragged_scene

pytestmark = pytest.mark.gpu


def _forward(ds, passes=L.SS_PASS_MAIN, opts=None, distortion=True):
    frame = Frame(ds.scene.cameras, passes, opts, distortion=distortion)
    out = frame.forward(ds.splats, ds.dF, ds.color)
    torch.cuda.synchronize()
    return frame, out


@pytest.mark.parametrize("name", list(SCENES))
def test_distortion_forward_parity(name):
    scene = SCENES[name]()
    ds = DeviceScene(scene)
    frame, out = _forward(ds)
    ora = oracle_forward(ds.stored_scene64(), scene.cameras[0])
    keep = ora["margin_fwd"] >= MARGIN
    err = np.abs(to_np(out.distort[0]) - ora["distort"])[keep].max()
    assert err <= FWD_TOL, err
    assert np.abs(ora["distort"]).max() > 1e-2
    # the other planes are those of the run without the distortion, bit for bit
    _, ref = _forward(ds, distortion=False)
    for k in ("rgb", "depth", "normal", "alpha", "T_final", "last"):
        assert torch.equal(getattr(ref, k)[0], getattr(out, k)[0]), k
    check_forward(gpu_planes(out, 0), ora, sun=False, tol=FWD_TOL)


@pytest.mark.parametrize("tile,batch,persistent", [((16, 16), 256, 1), ((32, 8), 256, 0), ((8, 32), 256, 1),
                                                   ((16, 16), 256, 0), ((32, 16), 256, 1)])
def test_distortion_tile_shapes_agree(tile, batch, persistent):
    scene = ragged_scene(seed=4)
    ds = DeviceScene(scene)
    _, ref = _forward(ds)
    opts = L.default_opts(tile_w=tile[0], tile_h=tile[1], batch=batch, persistent=persistent)
    _, out = _forward(ds, opts=opts)
    assert torch.equal(ref.distort[0], out.distort[0])


def _backward_case(ds, frame, out, seed, only_distort):
    s64 = ds.stored_scene64()
    rng = np.random.default_rng(seed)
    ups, ups_np = [], []
    for t in frame.targets:
        o = oracle_forward(s64, ds.scene.cameras[t.cam], sun=t.sun)
        m = (o["margin_bwd"] >= MARGIN).astype(np.float64)
        r, d, n, a = scenegen.upstream_grads(rng, t.height, t.width, sun=t.sun)
        u = dict(depth=d * m, alpha=a * m)
        if not t.sun:
            u.update(rgb=r * m, normal=n * m, distort=rng.normal(size=(t.height, t.width)) * m)
        if only_distort:
            u = {k: v for k, v in u.items() if k == "distort"}
        ups_np.append({k: np.asarray(v, np.float64) for k, v in u.items()})
        ups.append({k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda() for k, v in u.items()})
    # the upstream the oracle sees is the float32 one the kernels see
    ups_np = [{k: v.astype(np.float32).astype(np.float64) for k, v in u.items()} for u in ups_np]
    grads = zero_grads(ds.n_pad, "cuda")
    V = frame.n_cams
    d_dF = torch.zeros(V, 2, 4, device="cuda")
    d_col = torch.zeros(V, 3, 4, device="cuda")
    frame.backward(ds.splats, out, ups, grads, d_dF=d_dF, d_color=d_col)
    torch.cuda.synchronize()
    ref = None
    for t, u in zip(frame.targets, ups_np):
        cam = ds.scene.cameras[t.cam]
        r = oracle.backward(s64, cam, u, sun=t.sun, color=None if t.sun else cam.color)
        ref = r if ref is None else {k: ref[k] + r[k] for k in ref}
    n = ds.n
    for k in ("means", "scales", "quats", "opacity", "rgb"):
        g = to_np(grads[k][:, :n])
        if only_distort and k == "rgb":
            assert np.abs(g).max() == 0.0
            continue
        grad_close(g, ref[k].reshape(g.shape), name=k)
    grad_close(to_np(d_dF[0]), ref["dF"], name="dF")


@pytest.mark.parametrize("name,passes,only", [("small", L.SS_PASS_MAIN, True), ("ragged", L.SS_PASS_MAIN, False),
                                              ("ragged", 3, False)])
def test_distortion_backward_parity(name, passes, only):
    scene = SCENES[name]()
    for c in scene.cameras:
        c.shadow_w, c.shadow_h = 80, 64
    ds = DeviceScene(scene)
    frame, out = _forward(ds, passes=passes)
    _backward_case(ds, frame, out, seed=13, only_distort=only)


def test_distortion_adjoint_needs_the_depth_plane():
    scene = ragged_scene(seed=6)
    ds = DeviceScene(scene)
    frame, out = _forward(ds)
    io = out.io_array([dict(distort=torch.zeros_like(out.alpha[0]))])
    io[0].depth = None
    g = grads_struct(zero_grads(ds.n_pad, "cuda"))
    with pytest.raises(L.SatSplatError) as e:
        L.rasterize_bwd(ds.splats, frame.cams, frame.n_cams, frame.passes, frame.opts, io, g, None, None,
                        frame.ws, frame.ws_bytes, frame.capacity)
    assert e.value.status == L.SS_ERR_INVALID_ARG


def test_distortion_through_autograd_and_the_batched_step():
    """loss = sum W distort (+ the other planes) through the autograd form, and the batched
    graph step with the distortion, against the oracle."""
    from paper_2606_28581_gb300.autograd import render
    from paper_2606_28581_gb300.batched import BatchedStep

    scene = scenegen.make_scene(n=2500, extent_m=50.0, seed=41, views=[
        dict(width=72, height=60, off_nadir=16.0, delta=True, color_noise=0.02),
        dict(width=64, height=56, off_nadir=9.0, delta=True, color_noise=0.02)])
    s64 = oracle.SceneF64.of(scene)
    rng = np.random.default_rng(5)
    Ws, ref = [], None
    for cam in scene.cameras:
        o = oracle.render(s64, cam, color=cam.color)
        W = rng.normal(size=(cam.height, cam.width)) * (o["margin_bwd"] >= MARGIN)
        W = W.astype(np.float32).astype(np.float64)
        Ws.append(W)
        r = oracle.backward(s64, cam, dict(distort=W), color=cam.color)
        ref = r if ref is None else {k: ref[k] + r[k] for k in ref}
    # autograd form
    t = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda", requires_grad=True)
    P = dict(means=t(scene.means), scales=t(scene.scales), quats=t(scene.quats), opacity=t(scene.opacity),
             rgb=t(scene.rgb), dF=t(np.stack([c.dF_xy for c in scene.cameras])),
             color=t(np.stack([c.color for c in scene.cameras])))
    frame = Frame(scene.cameras, L.SS_PASS_MAIN, distortion=True)
    outs = render(frame, P["means"], P["scales"], P["quats"], P["opacity"], P["rgb"], P["dF"], P["color"])
    loss = sum((torch.from_numpy(W.astype(np.float32)).cuda() * o["distort"]).sum() for W, o in zip(Ws, outs))
    loss.backward()
    for k in ("means", "scales", "quats", "opacity"):
        grad_close(to_np(P[k].grad).reshape(-1), ref[k].reshape(-1), name=k)
    assert float(P["rgb"].grad.abs().max()) == 0.0
    # batched graph step (all views in one frame, upstream distortion only)
    n = scene.n
    ds = DeviceScene(scene)
    splats = dict(means=ds.means, scales=ds.scales, quats=ds.quats, opacity=ds.opacity, rgb=ds.rgb)
    ups = [dict(distort=torch.from_numpy(W.astype(np.float32)).cuda()) for W in Ws]
    step = BatchedStep(scene.cameras, splats, n, ds.dF, ds.color, ups, passes=L.SS_PASS_MAIN, distortion=True)
    step.capture()
    step.replay()
    torch.cuda.synchronize()
    for c, cam in enumerate(scene.cameras):
        o = oracle.render(s64, cam, color=cam.color)
        keep = o["margin_fwd"] >= MARGIN
        assert np.abs(to_np(step.out.distort[c]) - o["distort"])[keep].max() <= FWD_TOL
    for k in ("means", "scales", "quats", "opacity"):
        grad_close(to_np(step.grads[k][:, :n]).reshape(-1), ref[k].reshape(-1), name="batched " + k)
