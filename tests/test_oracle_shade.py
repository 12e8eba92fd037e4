"""Pins of the FP64 shading oracle (sun visibility and image formation), on the CPU.

Independent checks: the sun position against the renderer's own sun camera (Supp. A) applied to
the explicitly reconstructed 3-D receiver; closed forms for lit ground, a flat occluder and the
ambient limit; texel-centre sampling; and the hand-written adjoint against central differences."""
import numpy as np

import oracle
import scenegen
from oracle import shade as S

K, BIAS, EPS = 400.0, 0.0, 1e-3


def _cam(seed=0, w=48, h=40, off=20.0):
    sc = scenegen.make_scene(n=16, extent_m=80.0, seed=seed,
                             views=[dict(width=w, height=h, off_nadir=off, delta=True, shadow_scale=0.5)])
    return sc.cameras[0]


def test_sun_position_matches_the_sun_camera_on_the_reconstructed_point():
    cam = _cam(seed=3)
    rng = np.random.default_rng(0)
    H, W = cam.height, cam.width
    maxalt = float(np.float32(cam.max_alt))
    heights = rng.uniform(0.0, 0.04, size=(H, W))
    alpha = rng.uniform(0.5, 1.0, size=(H, W))
    depth = (maxalt - heights) * alpha
    ux, uy = S.sun_position(depth, alpha, cam, EPS)
    Bm, bm, _, _ = oracle.camera(cam, sun=False)
    Bs, bs, _, _ = oracle.camera(cam, sun=True)
    for (j, i) in [(0, 0), (5, 17), (H - 1, W - 1), (23, 3)]:
        x = np.array([i + 0.5, j + 0.5])
        hh = heights[j, i]
        XY = np.linalg.solve(Bm[:, :2], x - bm - Bm[:, 2] * hh)
        P = np.array([XY[0], XY[1], hh])
        u = Bs @ P + bs
        assert abs(u[0] - ux[j, i]) < 1e-9 and abs(u[1] - uy[j, i]) < 1e-9


def _planes(cam, heights, alpha, sun_heights, sun_alpha):
    maxalt = float(np.float32(cam.max_alt))
    return (maxalt - heights) * alpha, alpha, (maxalt - sun_heights) * sun_alpha, sun_alpha


def test_flat_lit_ground_is_fully_visible():
    cam = _cam(seed=1)
    H, W, Hs, Ws = cam.height, cam.width, cam.shadow_h, cam.shadow_w
    rng = np.random.default_rng(1)
    rgb = rng.uniform(0, 1, (3, H, W))
    d, a, sd, sa = _planes(cam, np.zeros((H, W)), np.full((H, W), 0.9), np.zeros((Hs, Ws)), np.full((Hs, Ws), 0.7))
    # a bias above the rounding of D / alpha makes exactly flat ground lit
    I, V = S.shade_forward(rgb, d, a, sd, sa, cam, [0.3, 0.4, 0.5], K, 1e-12, EPS)
    assert np.all(V == 1.0) and np.array_equal(I, rgb)


def test_flat_occluder_gives_the_closed_form_shadow():
    """Receivers on the ground, an occluder layer at height Ho over part of the sun view:
    pixels whose sun position falls well inside it get V = exp(-k (Ho - bias)); the rest are lit."""
    cam = _cam(seed=2, w=64, h=64)
    H, W, Hs, Ws = cam.height, cam.width, cam.shadow_h, cam.shadow_w
    Ho, bias = 0.003, 0.0005
    sun_h = np.zeros((Hs, Ws))
    sun_h[:, : Ws // 2] = Ho
    d, a, sd, sa = _planes(cam, np.zeros((H, W)), np.ones((H, W)), sun_h, np.ones((Hs, Ws)))
    La = [0.2, 0.3, 0.4]
    rgb = np.ones((3, H, W))
    I, V = S.shade_forward(rgb, d, a, sd, sa, cam, La, K, bias, EPS)
    ux, uy = S.sun_position(d, a, cam, EPS)
    inside = (ux > 1.5) & (ux < Ws / 2 - 1.5) & (uy > 1.5) & (uy < Hs - 1.5)
    lit = (ux > Ws / 2 + 1.5) & (ux < Ws - 1.5) & (uy > 1.5) & (uy < Hs - 1.5)
    assert inside.sum() > 50 and lit.sum() > 50
    vs = np.exp(-K * (Ho - bias))
    assert np.allclose(V[inside], vs, rtol=1e-12, atol=0)
    assert np.all(V[lit] == 1.0)
    for c in range(3):
        assert np.allclose(I[c][inside], La[c] + vs * (1 - La[c]), rtol=1e-12)


def test_deep_shadow_leaves_the_ambient_term():
    cam = _cam(seed=4)
    H, W, Hs, Ws = cam.height, cam.width, cam.shadow_h, cam.shadow_w
    d, a, sd, sa = _planes(cam, np.zeros((H, W)), np.ones((H, W)), np.full((Hs, Ws), 0.05), np.ones((Hs, Ws)))
    rgb = np.random.default_rng(4).uniform(0, 1, (3, H, W))
    La = np.array([0.25, 0.5, 0.75])
    I, V = S.shade_forward(rgb, d, a, sd, sa, cam, La, 5e3, 0.0, EPS)
    ux, uy = S.sun_position(d, a, cam, EPS)
    ok = (ux > 1) & (ux < Ws - 2) & (uy > 1) & (uy < Hs - 2)
    assert ok.sum() > 20
    assert np.allclose(I[:, ok], rgb[:, ok] * La[:, None], atol=1e-12)


def test_sampling_at_texel_centres_returns_the_texel():
    """A receiver whose sun position is exactly a texel centre compares against that texel alone."""
    cam = _cam(seed=5)
    H, W, Hs, Ws = cam.height, cam.width, cam.shadow_h, cam.shadow_w
    rng = np.random.default_rng(5)
    sun_h = rng.uniform(0.0, 0.01, (Hs, Ws))
    d, a, sd, sa = _planes(cam, np.zeros((H, W)), np.ones((H, W)), sun_h, np.ones((Hs, Ws)))
    g = S._geometry(d, a, sd, sa, cam, None, EPS)
    # the interpolant agrees with the texel value where the fractional offsets vanish
    fx = np.zeros_like(g["fx"]); fy = np.zeros_like(g["fy"])
    zs = g["zs"]
    zo0 = (1 - fx) * (1 - fy) * zs[g["jc"], g["ic"]]
    assert np.allclose(zo0, zs[g["jc"], g["ic"]])
    # and the bilinear weights of every sample sum to one
    assert np.allclose(sum(g["w"]), 1.0)


def _smooth(rng, shape, lo, hi, n=6):
    yy, xx = np.mgrid[0:shape[0], 0:shape[1]] / max(shape)
    f = np.zeros(shape)
    for _ in range(n):
        a, b, c = rng.normal(size=3)
        f += np.sin(3 * a * xx + 3 * b * yy + c)
    f = (f - f.min()) / (f.max() - f.min() + 1e-12)
    return lo + (hi - lo) * f


def test_adjoint_matches_central_differences():
    cam = _cam(seed=6, w=40, h=36)
    H, W, Hs, Ws = cam.height, cam.width, cam.shadow_h, cam.shadow_w
    rng = np.random.default_rng(6)
    heights = _smooth(rng, (H, W), 0.0, 0.004)
    alpha = _smooth(rng, (H, W), 0.6, 1.0)
    sun_h = _smooth(rng, (Hs, Ws), 0.0, 0.008)
    sun_a = _smooth(rng, (Hs, Ws), 0.6, 1.0)
    d, a, sd, sa = _planes(cam, heights, alpha, sun_h, sun_a)
    rgb = rng.uniform(0.1, 1.0, (3, H, W))
    La = np.array([0.3, 0.4, 0.5])
    dF = np.asarray(cam.dF_xy, np.float64)
    wI = rng.normal(size=(3, H, W))
    k = 300.0

    def loss(rgb_, d_, a_, sd_, sa_, La_, dF_):
        I, _ = S.shade_forward(rgb_, d_, a_, sd_, sa_, cam, La_, k, 0.0, EPS, dF=dF_)
        return float(np.sum(wI * I))

    g = S.shade_backward(wI, rgb, d, a, sd, sa, cam, La, k, 0.0, EPS, dF=dF)
    margin, frac = S.shade_margin(d, a, sd, sa, cam, k, 0.0, EPS, dF=dF)
    # directions that move no pixel across a decision (margins far above the step)
    keep = (margin > 1e-3) & (frac > 1e-3)
    assert keep.mean() > 0.9
    base = dict(rgb_=rgb, d_=d, a_=a, sd_=sd, sa_=sa, La_=La, dF_=dF)
    names = dict(rgb_="rgb", d_="depth", a_="alpha", sd_="sun_depth", sa_="sun_alpha", La_="La", dF_="dF")
    steps = dict(rgb_=1e-6, d_=1e-9, a_=1e-7, sd_=1e-9, sa_=1e-7, La_=1e-6, dF_=1e-6)
    for key, hstep in steps.items():
        dirn = rng.normal(size=np.shape(base[key]))
        if key in ("d_", "a_"):
            dirn = dirn * keep
        if key == "dF_":
            dirn[:, 3] = 0.0
        plus = dict(base); plus[key] = base[key] + hstep * dirn
        minus = dict(base); minus[key] = base[key] - hstep * dirn
        fd = (loss(**plus) - loss(**minus)) / (2 * hstep)
        an = float(np.sum(g[names[key]] * dirn))
        assert abs(fd - an) <= 1e-6 + 2e-3 * abs(an), (key, fd, an)
