"""The fused Adam step (with the 3DGS-MCMC position noise) and the 3DGS-MCMC relocation on the
GPU against the FP64 optimiser oracle, through the C ABI."""
import math

import numpy as np
import pytest
import torch

import scenegen
from oracle import optim as O
from paper_2606_28581_gb300 import _lib as L
from paper_2606_28581_gb300.frame import n_pad_of
from tests.gpu_util import to_np

pytestmark = pytest.mark.gpu

ROWS = O.PARAM_ROWS
GRAD_ROWS = {"means": 3, "scales": 2, "quats": 4, "opacity": 1, "rgb": 3}
STORE_OF = {"means": "means", "log_scales": "scales", "quats": "quats", "logit_opacity": "opacity", "rgb": "rgb"}
ULP32 = 2.0 ** -23


def _rand_params(rng, n_pad, n):
    """Raw parameters with opacities on both sides of the noise gate (o = 0.005) and small scales."""
    p = dict(means=rng.normal(0, 0.3, (3, n_pad)), log_scales=np.log(rng.uniform(1e-3, 4e-3, (2, n_pad))),
             quats=rng.normal(size=(4, n_pad)), logit_opacity=rng.normal(math.log(0.005 / 0.995), 2.5, (1, n_pad)),
             rgb=rng.uniform(0, 1, (3, n_pad)))
    return {k: a.astype(np.float32) for k, a in p.items()}


def _dev(d):
    return {k: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda() for k, a in d.items()}


def _params_struct(t):
    return L.make_params(t["means"], t["log_scales"], t["quats"], t["logit_opacity"], t["rgb"])


def _storage(n, n_pad, dtype):
    z = lambda c: torch.zeros(c, n_pad, device="cuda", dtype=dtype)
    st = dict(means=z(3), scales=z(2), quats=z(4), opacity=z(1), rgb=z(3))
    return st, L.make_splats(st["means"], st["scales"], st["quats"], st["opacity"], st["rgb"], n)


def _close_update(gpu, ora, before, name, rel=1e-5, per_column=False):
    """|gpu - oracle| <= 4 ulp(|oracle|) + rel |oracle - before| (FP32 rounding of the result and a
    relative error of the update); with per_column the update's scale is the largest change
    of the column (the three components of a position share one noise vector)."""
    d = np.abs(gpu - ora)
    delta = np.abs(ora - before)
    if per_column:
        delta = np.broadcast_to(delta.max(axis=0, keepdims=True), delta.shape)
    bound = 4 * ULP32 * np.abs(ora) + rel * delta + 1e-30
    bad = d > bound
    assert not bad.any(), f"{name}: {bad.sum()} elements out of bound; worst {d[bad].max():.3e}"


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_adam_step_matches_oracle(dtype):
    rng = np.random.default_rng(1 if dtype == torch.float32 else 2)
    n = 4997  # a ragged tail: the last thread owns one splat
    n_pad = n_pad_of(n)
    raw = _rand_params(rng, n_pad, n)
    m = {k: (rng.normal(size=a.shape) * 1e-2).astype(np.float32) for k, a in raw.items()}
    v = {k: (rng.uniform(size=a.shape) * 1e-4).astype(np.float32) for k, a in raw.items()}
    g = {k: rng.normal(size=(c, n_pad)).astype(np.float32) for k, c in GRAD_ROWS.items()}
    opts = L.default_adam_opts(step=7, seed=12345)
    lr = dict(means=opts.lr_means, log_scales=opts.lr_scales, quats=opts.lr_quats, logit_opacity=opts.lr_opacity,
              rgb=opts.lr_rgb)
    tp, tm, tv, tg = _dev(raw), _dev(m), _dev(v), _dev(g)
    st, storage = _storage(n, n_pad, dtype)
    grads = L.ss_splat_grads()
    grads.means, grads.scales, grads.quats, grads.opacity, grads.rgb = (L.ptr(tg[k]) for k in GRAD_ROWS)
    grads.n_pad = n_pad
    L.adam_step(_params_struct(tp), _params_struct(tm), _params_struct(tv), grads, storage, opts)
    torch.cuda.synchronize()
    f32 = lambda x: float(np.float32(x))
    sl = lambda d: {k: a[:, :n].astype(np.float64) for k, a in d.items()}
    ora, om, ov, ost = O.adam_step(sl(raw), sl(m), sl(v), sl(g), {k: f32(x) for k, x in lr.items()}, f32(opts.beta1),
                                   f32(opts.beta2), f32(opts.eps), 7, noise_lr=f32(opts.noise_lr),
                                   noise_k=f32(opts.noise_k), noise_t=f32(opts.noise_t), seed=12345)
    gate = 1 / (1 + np.exp(100 * (O.sigmoid(ora["logit_opacity"][0]) - 0.005)))
    assert (gate > 0.1).sum() > 500 and (gate < 1e-3).sum() > 500  # both sides of the gate
    for k in raw:
        gk = to_np(tp[k])
        _close_update(gk[:, :n], ora[k], raw[k][:, :n].astype(np.float64), "raw " + k, per_column=k == "means")
        np.testing.assert_array_equal(gk[:, n:], raw[k][:, n:].astype(np.float64))  # the padding is untouched
        _close_update(to_np(tm[k])[:, :n], om[k], m[k][:, :n].astype(np.float64), "m " + k)
        _close_update(to_np(tv[k])[:, :n], ov[k], v[k][:, :n].astype(np.float64), "v " + k)
        # the storage holds the activation of the GPU's own raw values (FP32, then rounded)
        act = O.activated({kk: to_np(tp[kk])[:, :n] for kk in raw})[STORE_OF[k]]
        sv = to_np(st[STORE_OF[k]])[:, :n]
        tol = 4 * ULP32 if dtype == torch.float32 else 2.0 ** -8
        assert np.all(np.abs(sv - act) <= tol * np.abs(act) + 1e-30), k


def test_adam_flat_matches_oracle():
    rng = np.random.default_rng(3)
    n = 16 * 12
    x, m, v, g = (rng.normal(size=n).astype(np.float32) for _ in range(4))
    v = np.abs(v) * 1e-3
    opts = L.default_adam_opts(step=4)
    t = [torch.from_numpy(a.copy()).cuda() for a in (x, m, v, g)]
    L.adam_flat(t[0], t[1], t[2], t[3], 1e-3, opts)
    torch.cuda.synchronize()
    f32 = lambda z: float(np.float32(z))
    ox, om, ov = O.adam_update(x.astype(np.float64), m.astype(np.float64), v.astype(np.float64),
                               g.astype(np.float64), f32(1e-3), f32(opts.beta1), f32(opts.beta2), f32(opts.eps), 4)
    _close_update(to_np(t[0]), ox, x.astype(np.float64), "x")
    _close_update(to_np(t[1]), om, m.astype(np.float64), "m")
    _close_update(to_np(t[2]), ov, v.astype(np.float64), "v")


def _relocation_state(rng, n, cap, dead_frac, dtype):
    n_pad = n_pad_of(cap)
    raw = _rand_params(rng, n_pad, n)
    raw["logit_opacity"][0] = rng.normal(0.0, 2.0, n_pad).astype(np.float32)
    dead = rng.uniform(size=n_pad) < dead_frac
    raw["logit_opacity"][0, dead] = -7.5
    m = {k: rng.normal(size=a.shape).astype(np.float32) for k, a in raw.items()}
    v = {k: rng.uniform(size=a.shape).astype(np.float32) for k, a in raw.items()}
    st, storage = _storage(n, n_pad, dtype)
    act = O.activated({k: a.astype(np.float64) for k, a in raw.items()})
    rnd = scenegen.to_bf16_exact if dtype == torch.bfloat16 else (lambda a: a)
    host = {k: rnd(a.astype(np.float32)) for k, a in act.items()}  # the stored values, rounded here
    for k in st:
        st[k].copy_(torch.from_numpy(host[k]).to(dtype))
    return raw, m, v, st, storage, n_pad, host["opacity"][0].astype(np.float64)


@pytest.mark.parametrize("dtype,n,cap,dead_frac", [(torch.float32, 5000, 6000, 0.08),
                                                   (torch.bfloat16, 5000, 5100, 0.08),
                                                   (torch.float32, 3001, 3001, 0.3)])
def test_mcmc_relocation_matches_oracle(dtype, n, cap, dead_frac):
    rng = np.random.default_rng(n + cap)
    raw, m, v, st, storage, n_pad, stored = _relocation_state(rng, n, cap, dead_frac, dtype)
    tp, tm, tv = _dev(raw), _dev(m), _dev(v)
    opts = L.default_mcmc_opts(step=9, seed=777)
    ws = torch.empty(L.mcmc_workspace_size(cap), dtype=torch.uint8, device="cuda")
    stats = torch.zeros(2, dtype=torch.int64, device="cuda")
    n_after = L.mcmc_relocate(_params_struct(tp), _params_struct(tm), _params_struct(tv), storage, cap, opts, ws,
                              d_stats=stats)
    torch.cuda.synchronize()
    ora, om, ov, o_after, info = O.relocate({k: a.astype(np.float64) for k, a in raw.items()},
                                            {k: a.astype(np.float64) for k, a in m.items()},
                                            {k: a.astype(np.float64) for k, a in v.items()}, stored, n, cap,
                                            float(np.float32(opts.min_opacity)), float(np.float32(opts.growth)),
                                            opts.n_max, 9, 777)
    assert n_after == o_after
    n_dead = int(sum(1 for x in stored[:n] if x <= np.float32(0.005)))
    W = sum(int(math.floor(x * 2 ** 24)) for x in stored[:n] if x > np.float32(0.005))
    assert stats.cpu().tolist() == [n_dead, W]
    assert len(info["targets"]) == n_dead + (n_after - n) > 0
    rewritten = np.zeros(n_pad, bool)
    rewritten[info["targets"]] = True
    sources = np.zeros(n_pad, bool)
    sources[list(info["counts"])] = True
    for k in raw:
        gk, ok = to_np(tp[k]), ora[k]
        # the new opacity and scales of the sources (and so of their copies) are computed in FP64
        # on both sides and rounded to FP32; every other value is copied or untouched: bit-exact
        split = (rewritten | sources) if k in ("log_scales", "logit_opacity") else np.zeros(n_pad, bool)
        np.testing.assert_array_equal(gk[:, ~split], ok[:, ~split].astype(np.float32).astype(np.float64), err_msg=k)
        d = np.abs(gk[:, split] - ok[:, split])
        assert np.all(d <= 2 * ULP32 * np.abs(ok[:, split]) + 1e-30), k
        reset = rewritten | sources
        for mom, om_ in ((tm, om), (tv, ov)):
            g_m = to_np(mom[k])
            assert np.all(g_m[:, reset] == 0.0)
            np.testing.assert_array_equal(g_m[:, ~reset], om_[k][:, ~reset].astype(np.float32).astype(np.float64))
    # the storage of every rewritten splat is the activation of its new raw values
    act = O.activated({k: to_np(tp[k]) for k in raw})
    tol = 4 * ULP32 if dtype == torch.float32 else 2.0 ** -8
    touched = rewritten | sources
    for k in st:
        sv = to_np(st[k])[:, touched]
        assert np.all(np.abs(sv - act[k][:, touched]) <= tol * np.abs(act[k][:, touched]) + 1e-30), k


def test_mcmc_without_live_splats_changes_nothing():
    rng = np.random.default_rng(9)
    raw, m, v, st, storage, n_pad, _ = _relocation_state(rng, 300, 400, 2.0, torch.float32)
    tp, tm, tv = _dev(raw), _dev(m), _dev(v)
    ws = torch.empty(L.mcmc_workspace_size(400), dtype=torch.uint8, device="cuda")
    n_after = L.mcmc_relocate(_params_struct(tp), _params_struct(tm), _params_struct(tv), storage, 400,
                              L.default_mcmc_opts(), ws)
    torch.cuda.synchronize()
    assert n_after == 300
    for k in raw:
        np.testing.assert_array_equal(to_np(tp[k]), raw[k].astype(np.float64))


def test_optimiser_rejects_bad_arguments():
    n, n_pad = 64, 64
    t = _dev({k: np.zeros((c, n_pad), np.float32) for k, c in ROWS.items()})
    p = _params_struct(t)
    st, storage = _storage(n, n_pad, torch.float32)
    grads = L.ss_splat_grads()
    g = _dev({k: np.zeros((c, n_pad), np.float32) for k, c in GRAD_ROWS.items()})
    grads.means, grads.scales, grads.quats, grads.opacity, grads.rgb = (L.ptr(g[k]) for k in GRAD_ROWS)
    grads.n_pad = n_pad
    with pytest.raises(L.SatSplatError):
        L.adam_step(p, p, p, grads, storage, L.default_adam_opts(step=0))
    with pytest.raises(L.SatSplatError):
        L.adam_step(p, p, p, grads, storage, L.default_adam_opts(beta2=1.0))
    ws = torch.empty(L.mcmc_workspace_size(n), dtype=torch.uint8, device="cuda")
    with pytest.raises(L.SatSplatError):  # a budget above the arrays' n_pad
        L.mcmc_relocate(p, p, p, storage, 1000, L.default_mcmc_opts(), ws)
    with pytest.raises(L.SatSplatError):
        L.mcmc_relocate(p, p, p, storage, n, L.default_mcmc_opts(n_max=52), ws)
    # no active splat: both calls succeed and change nothing
    before = {k: to_np(v) for k, v in t.items()}
    _, empty = _storage(0, n_pad, torch.float32)
    L.adam_step(p, p, p, grads, empty, L.default_adam_opts())
    assert L.mcmc_relocate(p, p, p, empty, n, L.default_mcmc_opts(), ws) == 0
    torch.cuda.synchronize()
    for k, v in t.items():
        np.testing.assert_array_equal(to_np(v), before[k])


def test_full_size_adam_and_relocation_1M():
    """The bench's optimiser workload: 1M splats, BF16 storage.  The Adam step is checked on 3000
    sampled splats (the oracle draws their noise with their own indices); the relocation (about
    5 % dead, 5 % growth under a budget of 1.05M) is checked on every splat."""
    rng = np.random.default_rng(11)
    n, cap = 1_000_000, 1_050_000
    n_pad = n_pad_of(cap)
    raw = _rand_params(rng, n_pad, n)
    m = {k: (rng.normal(size=a.shape) * 1e-2).astype(np.float32) for k, a in raw.items()}
    v = {k: (rng.uniform(size=a.shape) * 1e-4).astype(np.float32) for k, a in raw.items()}
    g = {k: rng.normal(size=(c, n_pad)).astype(np.float32) for k, c in GRAD_ROWS.items()}
    opts = L.default_adam_opts(step=3, seed=5)
    tp, tm, tv, tg = _dev(raw), _dev(m), _dev(v), _dev(g)
    st, storage = _storage(n, n_pad, torch.bfloat16)
    grads = L.ss_splat_grads()
    grads.means, grads.scales, grads.quats, grads.opacity, grads.rgb = (L.ptr(tg[k]) for k in GRAD_ROWS)
    grads.n_pad = n_pad
    L.adam_step(_params_struct(tp), _params_struct(tm), _params_struct(tv), grads, storage, opts)
    torch.cuda.synchronize()
    idx = np.sort(rng.choice(n, 3000, replace=False))
    f32 = lambda x: float(np.float32(x))
    lr = dict(means=f32(opts.lr_means), log_scales=f32(opts.lr_scales), quats=f32(opts.lr_quats),
              logit_opacity=f32(opts.lr_opacity), rgb=f32(opts.lr_rgb))
    sel = lambda d: {k: a[:, idx].astype(np.float64) for k, a in d.items()}
    ora, om, ov, _ = O.adam_step(sel(raw), sel(m), sel(v), sel(g), lr, f32(opts.beta1), f32(opts.beta2),
                                 f32(opts.eps), 3, noise_lr=f32(opts.noise_lr), noise_k=f32(opts.noise_k),
                                 noise_t=f32(opts.noise_t), seed=5, index=idx)
    for k in raw:
        _close_update(to_np(tp[k])[:, idx], ora[k], raw[k][:, idx].astype(np.float64), "raw " + k,
                      per_column=k == "means")
        _close_update(to_np(tm[k])[:, idx], om[k], m[k][:, idx].astype(np.float64), "m " + k)
    # relocation on a fresh host-drawn state (about 5 % of the splats dead) in the same buffers
    raw = _rand_params(rng, n_pad, n)
    raw["logit_opacity"][0] = rng.normal(0.0, 2.0, n_pad).astype(np.float32)
    raw["logit_opacity"][0, rng.uniform(size=n_pad) < 0.05] = -8.0
    m = {k: rng.normal(size=a.shape).astype(np.float32) for k, a in raw.items()}
    v = {k: rng.uniform(size=a.shape).astype(np.float32) for k, a in raw.items()}
    for src, dst in ((raw, tp), (m, tm), (v, tv)):
        for k in src:
            dst[k].copy_(torch.from_numpy(src[k]))
    stored_np = scenegen.to_bf16_exact(O.sigmoid(raw["logit_opacity"].astype(np.float64)).astype(np.float32))
    st["opacity"].copy_(torch.from_numpy(stored_np).to(torch.bfloat16))
    before = {k: a.astype(np.float64) for k, a in raw.items()}
    mb, vb = {k: a.astype(np.float64) for k, a in m.items()}, {k: a.astype(np.float64) for k, a in v.items()}
    stored = stored_np[0].astype(np.float64)
    ws = torch.empty(L.mcmc_workspace_size(cap), dtype=torch.uint8, device="cuda")
    mo = L.default_mcmc_opts(step=2, seed=8)
    n_after = L.mcmc_relocate(_params_struct(tp), _params_struct(tm), _params_struct(tv), storage, cap, mo, ws)
    torch.cuda.synchronize()
    new, nm, nv, o_after, info = O.relocate(before, mb, vb, stored, n, cap, f32(mo.min_opacity), f32(mo.growth),
                                            mo.n_max, 2, 8)
    assert n_after == o_after == cap and len(info["targets"]) > 90_000
    split = np.zeros(n_pad, bool)
    split[info["targets"]] = True
    split[list(info["counts"])] = True
    for k in raw:
        gk = to_np(tp[k])
        if k in ("log_scales", "logit_opacity"):
            np.testing.assert_array_equal(gk[:, ~split], new[k][:, ~split].astype(np.float32).astype(np.float64))
            assert np.all(np.abs(gk[:, split] - new[k][:, split]) <= 2 * ULP32 * np.abs(new[k][:, split]) + 1e-30)
        else:
            np.testing.assert_array_equal(gk, new[k].astype(np.float32).astype(np.float64), err_msg=k)
        np.testing.assert_array_equal(to_np(tm[k]), nm[k].astype(np.float32).astype(np.float64), err_msg=k)


def test_training_loop_reduces_the_loss():
    """A few dozen fused steps on a small scene (render, L2 loss on the colour, backward through the
    C ABI, Adam, one relocation): the optimiser, the relocation and the rasterizer work together."""
    import scenegen
    from paper_2606_28581_gb300.frame import Frame
    from paper_2606_28581_gb300.optim import SplatOptimizer
    from tests.gpu_util import DeviceScene

    scene = scenegen.make_scene(n=1500, extent_m=40.0, seed=51, views=[dict(width=64, height=64, off_nadir=10.0)])
    ds = DeviceScene(scene)
    frame = Frame(scene.cameras, L.SS_PASS_MAIN)
    target = frame.forward(ds.splats, ds.dF, ds.color).rgb[0].clone()
    rng = np.random.default_rng(52)
    rgb0 = np.clip(scene.rgb + rng.normal(0, 0.2, scene.rgb.shape), 0.01, 0.99)
    adam = L.default_adam_opts(lr_means=1e-4, lr_rgb=0.02, noise_lr=0.0)
    opt = SplatOptimizer(scene.means, scene.scales, scene.quats, scene.opacity, rgb0, cap=1600,
                         storage=torch.float32, adam=adam)
    losses = []
    for it in range(40):
        out = frame.forward(opt.splats, ds.dF, ds.color)
        diff = out.rgb[0] - target
        losses.append(float((diff * diff).sum()))
        opt.zero_grad()
        frame.backward(opt.splats, out, [dict(rgb=2 * diff)], opt.grads)
        opt.step()
        if it == 20:
            assert opt.relocate() >= 1500
    assert losses[-1] < 0.3 * losses[0], losses[::8]
