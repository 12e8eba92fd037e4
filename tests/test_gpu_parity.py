"""CUDA path vs the FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from paper_2606_28581_gb300 import _lib as L
from paper_2606_28581_gb300.frame import Frame, zero_grads
from tests.gpu_util import (BF16_TOL, FWD_TOL, MARGIN, DeviceScene, check_forward, grad_close,
                            oracle_forward, run_forward, to_np)

pytestmark = pytest.mark.gpu


def ragged_scene(seed=1, n=3000, w=100, h=75, delta=True, color_noise=0.02, off=20.0):
    return scenegen.make_scene(n=n, extent_m=80.0, seed=seed,
                               views=[dict(width=w, height=h, off_nadir=off, delta=delta,
                                           color_noise=color_noise)])


SCENES = {
    "small": lambda: scenegen.workload("small"),
    "ragged": lambda: ragged_scene(),
}


def gpu_planes(out, i):
    return dict(rgb=to_np(out.rgb[i]), depth=to_np(out.depth[i]), normal=to_np(out.normal[i]),
                alpha=to_np(out.alpha[i]), T=to_np(out.T_final[i]))


@pytest.mark.parametrize("name", list(SCENES))
def test_forward_parity_main(name):
    scene = SCENES[name]()
    ds = DeviceScene(scene)
    frame, out = run_forward(ds)
    s64 = ds.stored_scene64()
    cam = scene.cameras[0]
    ora = oracle_forward(s64, cam)
    errs, excl = check_forward(gpu_planes(out, 0), ora, sun=False, tol=FWD_TOL)
    print(name, errs, f"excluded {excl:.4%}")


@pytest.mark.parametrize("name", list(SCENES))
def test_forward_parity_sun(name):
    scene = SCENES[name]()
    for c in scene.cameras:
        c.shadow_w, c.shadow_h = 96, 80
    ds = DeviceScene(scene)
    frame, out = run_forward(ds, passes=L.SS_PASS_SUN)
    s64 = ds.stored_scene64()
    ora = oracle_forward(s64, scene.cameras[0], sun=True)
    g = dict(depth=to_np(out.depth[0]), alpha=to_np(out.alpha[0]))
    errs, excl = check_forward(g, ora, sun=True, tol=FWD_TOL)
    print(name, errs, f"excluded {excl:.4%}")


def test_shadow_depth_entry_point_matches_sun_pass():
    scene = ragged_scene(seed=3)
    ds = DeviceScene(scene)
    frame, out = run_forward(ds, passes=L.SS_PASS_SUN)
    cam = scene.cameras[0]
    depth = torch.empty(cam.shadow_h, cam.shadow_w, device="cuda")
    alpha = torch.empty_like(depth)
    T = torch.empty_like(depth)
    last = torch.empty(cam.shadow_h, cam.shadow_w, device="cuda", dtype=torch.int32)
    io = (L.ss_target_io * 1)()
    io[0].depth, io[0].alpha, io[0].T_final, io[0].last = L.ptr(depth), L.ptr(alpha), L.ptr(T), L.ptr(last)
    f2 = Frame(scene.cameras, L.SS_PASS_SUN)
    f2.ensure_workspace(ds.splats, frame.capacity)
    st, needed = L.shadow_depth(ds.splats, f2.cams, 1, ds.dF, f2.opts, io, f2.ws, f2.ws_bytes, f2.capacity)
    torch.cuda.synchronize()
    assert st == L.SS_OK and needed == frame.needed
    assert torch.equal(depth, out.depth[0]) and torch.equal(alpha, out.alpha[0])


def _upstream(scene, frame, seed, masks):
    rng = np.random.default_rng(seed)
    ups, ups_np = [], []
    for i, t in enumerate(frame.targets):
        r, d, n, a = scenegen.upstream_grads(rng, t.height, t.width, sun=t.sun)
        m = masks[i]
        u = dict(depth=d * m, alpha=a * m)
        if not t.sun:
            u.update(rgb=r * m, normal=n * m)
        ups_np.append({k: v.astype(np.float64) for k, v in u.items()})
        ups.append({k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda() for k, v in u.items()})
    return ups, ups_np


@pytest.mark.parametrize("name,passes", [("small", L.SS_PASS_MAIN), ("ragged", L.SS_PASS_MAIN),
                                         ("ragged", L.SS_PASS_SUN), ("ragged", 3)])
def test_backward_parity(name, passes):
    scene = SCENES[name]()
    for c in scene.cameras:
        c.shadow_w, c.shadow_h = 80, 64
    ds = DeviceScene(scene)
    frame, out = run_forward(ds, passes=passes)
    s64 = ds.stored_scene64()
    oras = [oracle_forward(s64, scene.cameras[t.cam], sun=t.sun) for t in frame.targets]
    masks = [(o["margin_bwd"] >= MARGIN).astype(np.float64) for o in oras]
    ups, ups_np = _upstream(scene, frame, 7, masks)
    grads = zero_grads(ds.n_pad, "cuda")
    d_dF = torch.zeros(1, 2, 4, device="cuda")
    d_col = torch.zeros(1, 3, 4, device="cuda")
    frame.backward(ds.splats, out, ups, grads, d_dF=d_dF, d_color=d_col)
    torch.cuda.synchronize()
    ref = None
    for t, u in zip(frame.targets, ups_np):
        cam = scene.cameras[t.cam]
        r = oracle.backward(s64, cam, u, sun=t.sun, color=None if t.sun else cam.color)
        ref = r if ref is None else {k: ref[k] + r[k] for k in ref}
    n = ds.n
    for k in ("means", "scales", "quats", "opacity", "rgb"):
        g = grads[k][:, :n].cpu().numpy().astype(np.float64)
        rr = ref[k].reshape(g.shape)
        if passes == L.SS_PASS_SUN and k == "rgb":
            assert np.abs(g).max() == 0.0
            continue
        grad_close(g, rr, name=k)
    grad_close(d_dF[0].cpu().numpy().astype(np.float64), ref["dF"], name="dF")
    if passes & L.SS_PASS_MAIN:
        grad_close(d_col[0].cpu().numpy().astype(np.float64), ref["color"], name="color")


def test_bf16_storage_parity():
    scene = ragged_scene(seed=5)
    ds = DeviceScene(scene, dtype=torch.bfloat16)
    frame, out = run_forward(ds)
    s64 = ds.stored_scene64()  # the BF16 values as stored
    ora = oracle_forward(s64, scene.cameras[0])
    errs, _ = check_forward(gpu_planes(out, 0), ora, sun=False, tol=BF16_TOL)
    # storage error against the FP32 masters: information, reported not asserted
    ora32 = oracle_forward(oracle.SceneF64.of(scene), scene.cameras[0])
    storage = {k: float(np.abs(gpu_planes(out, 0)[k] - ora32[k]).max()) for k in ("rgb", "depth", "alpha")}
    print("bf16 errs", errs, "storage error vs fp32 masters", storage)


def test_bf16_backward_parity():
    scene = ragged_scene(seed=6)
    ds = DeviceScene(scene, dtype=torch.bfloat16)
    frame, out = run_forward(ds)
    s64 = ds.stored_scene64()
    cam = scene.cameras[0]
    ora = oracle_forward(s64, cam)
    ups, ups_np = _upstream(scene, frame, 9, [(ora["margin_bwd"] >= MARGIN).astype(np.float64)])
    grads = zero_grads(ds.n_pad, "cuda")
    d_dF = torch.zeros(1, 2, 4, device="cuda")
    frame.backward(ds.splats, out, ups, grads, d_dF=d_dF)
    ref = oracle.backward(s64, cam, ups_np[0], color=cam.color)
    for k in ("means", "scales", "quats", "opacity", "rgb"):
        g = grads[k][:, : ds.n].cpu().numpy().astype(np.float64)
        grad_close(g, ref[k].reshape(g.shape), name=k)
    grad_close(d_dF[0].cpu().numpy().astype(np.float64), ref["dF"], name="dF")


@pytest.mark.parametrize("tile,batch,persistent", [((32, 8), 256, 0), ((8, 32), 256, 0), ((16, 16), 256, 1),
                                                   ((32, 8), 256, 1), ((8, 32), 256, 1), ((32, 16), 256, 0),
                                                   ((16, 32), 256, 1)])
def test_tile_shape_and_schedule_do_not_change_outputs(tile, batch, persistent):
    scene = ragged_scene(seed=2)
    ds = DeviceScene(scene)
    _, ref = run_forward(ds, passes=3)
    opts = L.default_opts(tile_w=tile[0], tile_h=tile[1], batch=batch, persistent=persistent)
    _, out = run_forward(ds, passes=3, opts=opts)
    for i in range(2):
        for k in ("rgb", "depth", "normal", "alpha", "T_final"):
            a, b = getattr(ref, k)[i], getattr(out, k)[i]
            if a is None:
                continue
            assert torch.equal(a, b), (k, i)


def needle_scene(seed=3):
    """Footprints that stress the sub-block culling: a third of the splats are needles (one scale
    down to 1e-4 of the other), a third take any orientation, edge-on included."""
    scene = ragged_scene(seed=seed, n=4000, w=130, h=90)
    rng = np.random.default_rng(seed + 100)
    k = rng.permutation(scene.n)
    a, b = k[: scene.n // 3], k[scene.n // 3: 2 * scene.n // 3]
    scene.scales[1, a] = (scene.scales[1, a] * 10.0 ** rng.uniform(-4.0, -1.0, a.size)).astype(np.float32)
    q = rng.normal(size=(4, b.size))
    scene.quats[:, b] = (q / np.linalg.norm(q, axis=0)).astype(np.float32)
    scene.scales[:, b] = (scene.scales[:, b] * 3.0).astype(np.float32)
    return scene


@pytest.mark.parametrize("tile", [(16, 16), (32, 8), (8, 32), (32, 16), (16, 32)])
def test_subblock_culling_changes_nothing(tile):
    """The per-splat sub-block masks are conservative: walking every staged splat in every
    sub-block gives bitwise-identical forward outputs and the same gradients."""
    scene = needle_scene()
    for c in scene.cameras:
        c.shadow_w, c.shadow_h = 90, 70
    ds = DeviceScene(scene)
    runs = []
    for cull in (1, 0):
        opts = L.default_opts(tile_w=tile[0], tile_h=tile[1], subblock_cull=cull)
        frame, out = run_forward(ds, passes=3, opts=opts)
        ups = []
        rng = np.random.default_rng(11)
        for t in frame.targets:
            r, d, n, a = scenegen.upstream_grads(rng, t.height, t.width, sun=t.sun)
            u = dict(depth=d, alpha=a) if t.sun else dict(rgb=r, depth=d, normal=n, alpha=a)
            ups.append({k2: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda() for k2, v in u.items()})
        grads = zero_grads(ds.n_pad, "cuda")
        frame.backward(ds.splats, out, ups, grads)
        torch.cuda.synchronize()
        runs.append((out, grads))
    (o1, g1), (o0, g0) = runs
    for i in range(2):
        for k in ("rgb", "depth", "normal", "alpha", "T_final"):
            a, b = getattr(o1, k)[i], getattr(o0, k)[i]
            if a is not None:
                assert torch.equal(a, b), (k, i)
    # the per-pixel terms are bitwise equal; only the order of the atomic sums differs, which the
    # needles' large, cancelling per-pair terms make visible at ~1e-5 of the largest gradient
    for k in g1:
        grad_close(g0[k][:, :ds.n].cpu().numpy().astype(np.float64),
                   g1[k][:, :ds.n].cpu().numpy().astype(np.float64), name=k)


def test_needle_scene_forward_parity():
    """Thin and edge-on footprints against the oracle (the culled path)."""
    scene = needle_scene(seed=5)
    ds = DeviceScene(scene)
    frame, out = run_forward(ds, passes=1)
    ora = oracle_forward(ds.stored_scene64(), scene.cameras[0])
    check_forward(gpu_planes(out, 0), ora, sun=False, tol=FWD_TOL)


def test_batched_frame_equals_single_view_calls():
    scene = scenegen.make_scene(n=2500, extent_m=80.0, seed=4, views=[
        dict(width=96, height=64, off_nadir=10.0, delta=True, color_noise=0.02),
        dict(width=70, height=90, off_nadir=25.0, delta=True, color_noise=0.02),
        dict(width=128, height=40, off_nadir=15.0, delta=True)])
    ds = DeviceScene(scene)
    opts = L.default_opts(persistent=1)
    frame, out = run_forward(ds, passes=3, opts=opts)
    for c in range(3):
        sub = DeviceScene(scene)
        sub.dF = ds.dF[c:c + 1].contiguous()
        sub.color = ds.color[c:c + 1].contiguous()
        _, o1 = run_forward(sub, passes=3, cams=[scene.cameras[c]])
        for k in ("rgb", "depth", "normal", "alpha"):
            assert torch.equal(getattr(out, k)[c], getattr(o1, k)[0]), (c, k)
        assert torch.equal(out.depth[3 + c], o1.depth[1]) and torch.equal(out.alpha[3 + c], o1.alpha[1])


def test_targets_without_overlaps_between_others():
    """The tile sort orders each target's overlaps on its own: a view (and its sun view) that sees
    no splat, between views that do, leaves empty segments that change nothing elsewhere."""
    scene = scenegen.make_scene(n=2500, extent_m=80.0, seed=14, views=[
        dict(width=96, height=64, off_nadir=10.0, delta=True, color_noise=0.02),
        dict(width=70, height=90, off_nadir=25.0, delta=True, color_noise=0.02),
        dict(width=128, height=40, off_nadir=15.0, delta=True)])
    scene.cameras[1].F_xy[0, 3] += np.float32(1e5)  # the middle view looks far off the scene
    ds = DeviceScene(scene)
    frame, out = run_forward(ds, passes=3, opts=L.default_opts(persistent=1))
    assert torch.all(out.alpha[1] == 0) and torch.all(out.alpha[4] == 0)
    for c in (0, 2):
        sub = DeviceScene(scene)
        sub.dF = ds.dF[c:c + 1].contiguous()
        sub.color = ds.color[c:c + 1].contiguous()
        _, o1 = run_forward(sub, passes=3, cams=[scene.cameras[c]])
        assert torch.any(o1.alpha[0] > 0)
        for k in ("rgb", "depth", "normal", "alpha"):
            assert torch.equal(getattr(out, k)[c], getattr(o1, k)[0]), (c, k)
        assert torch.equal(out.depth[3 + c], o1.depth[1]) and torch.equal(out.alpha[3 + c], o1.alpha[1])


def test_capacity_overflow_is_reported_and_recovered():
    scene = ragged_scene(seed=8)
    ds = DeviceScene(scene)
    frame = Frame(scene.cameras, L.SS_PASS_MAIN, capacity=100)
    frame.ensure_workspace(ds.splats, 100)
    L.project_splats(ds.splats, frame.cams, 1, 1, ds.dF, ds.color, frame.opts, frame.ws, frame.ws_bytes, 100)
    st, needed = L.bin_and_sort(ds.splats, frame.cams, 1, 1, frame.opts, frame.ws, frame.ws_bytes, 100)
    assert st == L.SS_ERR_CAPACITY and needed > 100
    st2, needed2, _, _, flags = frame.status()
    assert st2 == L.SS_ERR_CAPACITY and needed2 == needed and flags & 1
    # the frame grows its workspace and re-runs
    out = frame.forward(ds.splats, ds.dF, ds.color)
    _, ref = run_forward(ds)
    assert frame.needed == needed and torch.equal(out.rgb[0], ref.rgb[0])


def test_invalid_arguments_are_rejected():
    scene = ragged_scene(seed=9)
    ds = DeviceScene(scene)
    frame = Frame(scene.cameras)
    frame.ensure_workspace(ds.splats, 1 << 16)
    lib = L.load()
    import ctypes
    bad = L.default_opts(tile_w=12)
    st = lib.ss_project_splats(ctypes.byref(ds.splats), frame.cams, 1, 1, None, None, ctypes.byref(bad),
                               L.ptr(frame.ws), frame.ws_bytes, frame.capacity, None)
    assert st == L.SS_ERR_INVALID_ARG
    st = lib.ss_project_splats(ctypes.byref(ds.splats), frame.cams, 1, 1, None, None, ctypes.byref(frame.opts),
                               L.ptr(frame.ws), 16, frame.capacity, None)
    assert st == L.SS_ERR_INVALID_ARG
    st = lib.ss_project_splats(ctypes.byref(ds.splats), frame.cams, 0, 1, None, None, ctypes.byref(frame.opts),
                               L.ptr(frame.ws), frame.ws_bytes, frame.capacity, None)
    assert st == L.SS_ERR_INVALID_ARG
    s2 = L.make_splats(ds.means, ds.scales, ds.quats, ds.opacity, ds.rgb, ds.n)
    s2.n_pad = ds.n_pad + 3
    st = lib.ss_project_splats(ctypes.byref(s2), frame.cams, 1, 1, None, None, ctypes.byref(frame.opts),
                               L.ptr(frame.ws), frame.ws_bytes, frame.capacity, None)
    assert st == L.SS_ERR_INVALID_ARG
    io = (L.ss_target_io * 1)()  # T_final / last missing
    st = lib.ss_rasterize_fwd(ctypes.byref(ds.splats), frame.cams, 1, 1, ctypes.byref(frame.opts), io,
                              L.ptr(frame.ws), frame.ws_bytes, frame.capacity, None)
    assert st == L.SS_ERR_INVALID_ARG


def test_nonfinite_splat_is_culled_and_counted():
    scene = ragged_scene(seed=10)
    ds = DeviceScene(scene)
    _, ref = run_forward(ds)
    # append a NaN splat: the image must not change
    sc2 = scenegen.Scene(*(np.concatenate([a, a[..., :1]], -1) for a in
                           (scene.means, scene.scales, scene.quats, scene.opacity, scene.rgb)),
                         cameras=scene.cameras, scale_m=scene.scale_m)
    sc2.means[0, -1] = np.nan
    ds2 = DeviceScene(sc2)
    frame, out = run_forward(ds2)
    st, _, nonfinite, _, _ = frame.status()
    assert st == L.SS_ERR_NONFINITE and nonfinite == 1
    assert torch.equal(out.rgb[0], ref.rgb[0])


def test_empty_scene():
    scene = ragged_scene(seed=11, n=8)
    scene.opacity[:] = 1e-3  # below 1/255: every splat is culled
    ds = DeviceScene(scene)
    frame, out = run_forward(ds)
    assert frame.needed == 0
    assert torch.all(out.alpha[0] == 0) and torch.all(out.T_final[0] == 1)
    c = torch.from_numpy(scene.cameras[0].color[:, 3]).cuda()
    assert torch.allclose(out.rgb[0], c[:, None, None].expand_as(out.rgb[0]))


def test_walked_pair_counter_matches_oracle():
    """The forward's count of walked (pixel, splat) pairs is the per-pixel contributor count
    of the definition (plus the stopping pair), summed over the image."""
    scene = ragged_scene(seed=12)
    ds = DeviceScene(scene)
    frame, out = run_forward(ds, opts=L.default_opts(count_pairs=1))
    _, _, _, walked, _ = frame.status()
    # without the option the forward does not count
    frame0, _ = run_forward(ds)
    assert frame0.status()[3] == 0
    ora = oracle_forward(ds.stored_scene64(), scene.cameras[0])
    ref = int(ora["ncontrib"].sum() + ora["terminated"].sum())
    slack = int((ora["margin_fwd"] < MARGIN).sum()) * 2
    assert abs(walked - ref) <= slack, (walked, ref)
