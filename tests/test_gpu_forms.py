"""The training forms: autograd wrapper (a), batched persistent step in a CUDA graph with the
autotuner (b), BF16 storage (c)."""
import os

import numpy as np
import pytest
import torch

import oracle
import scenegen
from paper_2606_28581_gb300 import _lib as L
from paper_2606_28581_gb300.autograd import render
from paper_2606_28581_gb300.batched import BatchedStep, autotune
from paper_2606_28581_gb300.frame import Frame
from tests.gpu_util import MARGIN, DeviceScene, grad_close, oracle_forward

pytestmark = pytest.mark.gpu


def scene3(seed=4, n=2500):
    return scenegen.make_scene(n=n, extent_m=80.0, seed=seed, views=[
        dict(width=96, height=64, off_nadir=10.0, delta=True, color_noise=0.02, shadow_scale=0.5),
        dict(width=70, height=90, off_nadir=25.0, delta=True, color_noise=0.02, shadow_scale=0.5),
        dict(width=128, height=40, off_nadir=15.0, delta=True, shadow_scale=0.5)])


def masters(scene):
    t = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda", requires_grad=True)
    return dict(means=t(scene.means), scales=t(scene.scales), quats=t(scene.quats), opacity=t(scene.opacity),
                rgb=t(scene.rgb),
                dF=t(np.stack([c.dF_xy for c in scene.cameras])), color=t(np.stack([c.color for c in scene.cameras])))


def weights(frame, scene, seed, s64):
    """Random upstream weights, zero at margin pixels (oracle decision margins)."""
    rng = np.random.default_rng(seed)
    ws = []
    for t in frame.targets:
        o = oracle_forward(s64, scene.cameras[t.cam], sun=t.sun)
        m = (o["margin_bwd"] >= MARGIN).astype(np.float32)
        r, d, n, a = scenegen.upstream_grads(rng, t.height, t.width, sun=t.sun)
        w = dict(depth=d * m, alpha=a * m)
        if not t.sun:
            w.update(rgb=r * m, normal=n * m)
        ws.append({k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda() for k, v in w.items()})
    return ws


def loss_of(outs, ws):
    return sum((o[k] * w[k]).sum() for o, w in zip(outs, ws) for k in w)


def loss64(outs, ws):
    """The same loss accumulated in float64 (finite differences need it)."""
    return sum(float((o[k].double() * w[k].double()).sum()) for o, w in zip(outs, ws) for k in w)


@pytest.mark.parametrize("storage", [torch.float32, torch.bfloat16])
def test_autograd_matches_oracle_adjoint(storage):
    scene = scene3()
    P = masters(scene)
    frame = Frame(scene.cameras, L.SS_PASS_MAIN | L.SS_PASS_SUN)
    # the oracle sees exactly the stored values (rounded to BF16 here, on the host)
    rnd = scenegen.to_bf16_exact if storage == torch.bfloat16 else (lambda a: a)
    st = {k: rnd(np.asarray(getattr(scene, k), np.float32)).astype(np.float64)
          for k in ("means", "scales", "quats", "opacity", "rgb")}
    s64 = oracle.SceneF64(st["means"], st["scales"], st["quats"], st["opacity"], st["rgb"])
    ws = weights(frame, scene, 3, s64)
    outs = render(frame, P["means"], P["scales"], P["quats"], P["opacity"], P["rgb"], P["dF"], P["color"],
                  storage=storage)
    loss_of(outs, ws).backward()
    ref = None
    for t, w in zip(frame.targets, ws):
        cam = scene.cameras[t.cam]
        u = {k: v.cpu().numpy().astype(np.float64) for k, v in w.items()}
        r = oracle.backward(s64, cam, u, sun=t.sun, color=None if t.sun else cam.color)
        r["dF_all"] = np.zeros((3, 2, 4)); r["dF_all"][t.cam] = r["dF"]
        r["col_all"] = np.zeros((3, 3, 4)); r["col_all"][t.cam] = r["color"]
        ref = r if ref is None else {k: ref[k] + r[k] for k in ref}
    for k in ("means", "scales", "quats", "opacity", "rgb"):
        g = P[k].grad.cpu().numpy().astype(np.float64)
        grad_close(g, ref[k].reshape(g.shape), name=k)
    grad_close(P["dF"].grad.cpu().numpy().astype(np.float64), ref["dF_all"], name="dF")
    grad_close(P["color"].grad.cpu().numpy().astype(np.float64), ref["col_all"], name="color")


def test_autograd_matches_central_differences():
    """Directional derivative of the loss through the GPU forward (FP32) by central
    differences against the autograd gradient; pixels near a threshold carry no weight."""
    scene = scenegen.make_scene(n=400, extent_m=40.0, seed=21, views=[
        dict(width=48, height=40, off_nadir=18.0, delta=True, color_noise=0.02)])
    P = masters(scene)
    frame = Frame(scene.cameras, L.SS_PASS_MAIN)
    s64 = oracle.SceneF64.of(scene)
    rng = np.random.default_rng(5)
    o = oracle_forward(s64, scene.cameras[0])
    m = (o["margin_bwd"] >= 2e-2).astype(np.float32)
    r, d, n, a = scenegen.upstream_grads(rng, 40, 48)
    ws = [{k: torch.from_numpy(np.ascontiguousarray(v * m, np.float32)).cuda()
           for k, v in dict(rgb=r, depth=d, normal=n, alpha=a).items()}]
    outs = render(frame, P["means"], P["scales"], P["quats"], P["opacity"], P["rgb"], P["dF"], P["color"])
    loss_of(outs, ws).backward()
    # perturbations of ~1e-3 px in screen position, ~0.1 % in size, ~1e-4 rad in orientation:
    # small enough that no weighted pixel crosses the 1/255 threshold (margin mask 2e-2)
    scale = dict(means=3e-5, scales=2e-5, quats=1e-4, opacity=5e-4, rgb=5e-4, dF=np.array([1e-3] * 3 + [1e-3]),
                 color=5e-4)
    dirs = {}
    for k, v in P.items():
        dk = rng.normal(size=tuple(v.shape)) * (scale[k] if k != "dF" else scale[k][None, None, :])
        dirs[k] = torch.from_numpy(dk.astype(np.float32)).cuda()
    analytic = sum(float((P[k].grad * dirs[k]).sum()) for k in P)

    def f(h):
        with torch.no_grad():
            q = {k: (P[k] + h * dirs[k]).contiguous() for k in P}
            fr = Frame(scene.cameras, L.SS_PASS_MAIN)
            outs = render(fr, q["means"], q["scales"], q["quats"], q["opacity"], q["rgb"], q["dF"], q["color"])
            return loss64(outs, ws)

    fd = (f(1.0) - f(-1.0)) / 2.0
    assert abs(fd - analytic) <= 2e-2 * max(abs(analytic), 1e-3), (fd, analytic)


def test_batched_graph_replay_matches_eager_and_oracle():
    scene = scene3(seed=7)
    ds = DeviceScene(scene, dtype=torch.bfloat16)
    frame0 = Frame(scene.cameras, 3)
    rng = np.random.default_rng(1)
    ups = []
    for t in frame0.targets:
        r, d, n, a = scenegen.upstream_grads(rng, t.height, t.width, sun=t.sun)
        u = dict(depth=d, alpha=a) if t.sun else dict(rgb=r, depth=d, normal=n, alpha=a)
        ups.append({k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in u.items()})
    splats = dict(means=ds.means, scales=ds.scales, quats=ds.quats, opacity=ds.opacity, rgb=ds.rgb)
    step = BatchedStep(scene.cameras, splats, ds.n, ds.dF, ds.color, ups)
    step.step_eager()
    torch.cuda.synchronize()
    eager = {k: v.clone() for k, v in step.grads.items()}
    eager_rgb = [x.clone() if x is not None else None for x in step.out.rgb]
    step.capture()
    for _ in range(2):
        step.replay()
    torch.cuda.synchronize()
    st, needed, walked, flags = step.check()
    assert st == L.SS_OK and flags == 0 and needed > 0 and walked == 0  # the step does not count
    assert step.count_walked() > 0
    for a, b in zip(eager_rgb, step.out.rgb):
        if a is not None:
            assert torch.equal(a, b)
    for k in eager:
        # the same sums in another atomic order
        grad_close(step.grads[k].cpu().numpy().astype(np.float64), eager[k].cpu().numpy().astype(np.float64),
                   rtol=1e-4, name=k)
    # the single-view plain path gives the same forward as the batched persistent launch
    frame1 = Frame([scene.cameras[1]], 3)
    sub = DeviceScene(scene, dtype=torch.bfloat16)
    out1 = frame1.forward(sub.splats, ds.dF[1:2].contiguous(), ds.color[1:2].contiguous())
    torch.cuda.synchronize()
    assert torch.equal(out1.rgb[0], step.out.rgb[1]) and torch.equal(out1.depth[1], step.out.depth[4])


def test_replay_from_host_matches_device_replay():
    """The host-buffer step (side-stream upload of the upstream planes) gives the same results as
    the device-resident replay, and changing the host inputs changes the results."""
    scene = scene3(seed=10)
    ds = DeviceScene(scene, dtype=torch.bfloat16)
    frame0 = Frame(scene.cameras, 3)
    rng = np.random.default_rng(2)
    ups = []
    for t in frame0.targets:
        r, d, n, a = scenegen.upstream_grads(rng, t.height, t.width, sun=t.sun)
        u = dict(depth=d, alpha=a) if t.sun else dict(rgb=r, depth=d, normal=n, alpha=a)
        ups.append({k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in u.items()})
    splats = dict(means=ds.means, scales=ds.scales, quats=ds.quats, opacity=ds.opacity, rgb=ds.rgb)
    step = BatchedStep(scene.cameras, splats, ds.n, ds.dF, ds.color, ups)
    step.capture()
    step.replay()
    torch.cuda.synchronize()
    ref = {k: v.clone() for k, v in step.grads.items()}
    ref_rgb = step.out.rgb[0].clone()
    pin = lambda t: t.detach().cpu().pin_memory()
    h_s = {k: pin(v) for k, v in splats.items()}
    h_u = [{k: pin(v) for k, v in u.items()} for u in ups]
    h_g = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in step.grads.items()}
    h_df = torch.empty_like(step.d_dF, device="cpu").pin_memory()
    # scramble the device copies: the host step must restore them
    for t in list(splats.values()) + [x for u in ups for x in u.values()]:
        t.zero_()
    step.replay_from_host(h_s, pin(ds.dF), pin(ds.color), h_u, h_g, h_df)
    torch.cuda.synchronize()
    assert torch.equal(step.out.rgb[0], ref_rgb)
    for k in ref:
        grad_close(h_g[k].numpy().astype(np.float64), ref[k].cpu().numpy().astype(np.float64), rtol=1e-4, name=k)
    assert torch.equal(h_df, step.d_dF.cpu())
    # new upstream values on the host reach the backward
    for u in h_u:
        for v in u.values():
            v.mul_(2.0)
    step.replay_from_host(h_s, pin(ds.dF), pin(ds.color), h_u, h_g)
    torch.cuda.synchronize()
    grad_close(h_g["rgb"].numpy().astype(np.float64), 2.0 * ref["rgb"].cpu().numpy().astype(np.float64),
               rtol=1e-4, name="rgb x2")


def test_batched_capacity_overflow_flag_after_replay():
    scene = scene3(seed=8)
    ds = DeviceScene(scene)
    frame0 = Frame(scene.cameras, 3)
    ups = [dict(depth=torch.ones(t.height, t.width, device="cuda")) for t in frame0.targets]
    splats = dict(means=ds.means, scales=ds.scales, quats=ds.quats, opacity=ds.opacity, rgb=ds.rgb)
    step = BatchedStep(scene.cameras, splats, ds.n, ds.dF, ds.color, ups, capacity=1000)
    step.capture()
    step.replay()
    st, needed, _, flags = step.check()
    assert st == L.SS_ERR_CAPACITY and flags & 1 and needed > step.frame.capacity


def test_autotuner_picks_and_caches(tmp_path):
    os.environ["SATSPLAT_AUTOTUNE_CACHE"] = str(tmp_path / "tune.json")
    try:
        scene = scene3(seed=9)
        ds = DeviceScene(scene)
        frame0 = Frame(scene.cameras, 3)
        ups = [dict(depth=torch.ones(t.height, t.width, device="cuda")) for t in frame0.targets]
        splats = dict(means=ds.means, scales=ds.scales, quats=ds.quats, opacity=ds.opacity, rgb=ds.rgb)
        mk = lambda o: BatchedStep(scene.cameras, splats, ds.n, ds.dF, ds.color, ups, opts=o)
        cands = [(16, 16, 256, 4), (8, 32, 256, 4)]
        opts, entry = autotune(mk, "test-key", candidates=cands)
        assert (opts.tile_w, opts.tile_h, opts.batch, opts.pixels_per_thread) in cands and opts.persistent == 1
        assert len(entry["ms"]) == 2
        opts2, entry2 = autotune(mk, "test-key", candidates=cands)
        assert entry2["best"] == entry["best"]
    finally:
        del os.environ["SATSPLAT_AUTOTUNE_CACHE"]
