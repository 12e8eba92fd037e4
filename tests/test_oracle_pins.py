"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
closed forms of the paper's equations, 3-D ray-plane geometry, library routines
(scipy's quaternion rotation), invariants of alpha compositing, brute force,
and forward-mode (dual number) and finite-difference derivatives."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from tests import helpers as H

OPT = oracle.Opts()
AMIN, AMAX, TMIN, SIG = OPT.alpha_min, OPT.alpha_max, OPT.t_min, OPT.sigma


def rot(q_wxyz):
    q = np.asarray(q_wxyz, np.float64)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy: (x, y, z, w)


def geometric_pixel(p, su, sv, q_wxyz, o, B, b, max_alt, px, py):
    """Ray-splat intersection by 3-D geometry: the pixel's ray is the line of world points
    that B maps to (px, py); intersect it with the splat plane.  Returns the lower-bounded
    Gaussian alpha (before the 1/255 test) and the depth of the intersection point."""
    R = rot(q_wxyz)
    tu, tv = R[:, 0], R[:, 1]
    d = np.cross(B[0], B[1])                 # direction along which B is constant
    p0 = np.linalg.lstsq(B, np.array([px, py]) - b, rcond=None)[0]
    A = np.stack([su * tu, sv * tv, -d], 1)
    u, v, t = np.linalg.solve(A, p0 - p)
    hit = p0 + t * d
    c = B @ p + b
    gu = math.exp(-0.5 * (u * u + v * v))
    gs = math.exp(-((px - c[0]) ** 2 + (py - c[1]) ** 2) / (2 * SIG * SIG))
    alpha = min(AMAX, o * max(gu, gs))
    return alpha, max_alt - hit[2], u, v


def one_splat_scene(cam, p, su, sv, q, o, rgb):
    return H.make(np.reshape(p, (3, 1)), [su, sv], np.reshape(q, (4, 1)), [o],
                  np.reshape(rgb, (3, 1)), [cam])


# ------------------------------------------------------------------------------ closed forms
@pytest.mark.parametrize("seed", range(6))
def test_single_splat_matches_ray_plane_geometry(seed):
    """Sec. 3.2 Eq. affine2dgs_Qq and Eq. depth_affine_camera against 3-D geometry."""
    rng = np.random.default_rng(100 + seed)
    cam = H.oblique_camera(rng, width=48, height=40, k=25.0, off_nadir_deg=rng.uniform(0, 35),
                           max_alt=1.5)
    p = np.array([rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), rng.uniform(0, 0.4)])
    q = H.quat_axis_angle(rng.normal(size=3), rng.uniform(0, 0.9)) * rng.uniform(0.5, 2)
    su, sv = rng.uniform(0.05, 0.2, 2)
    o = rng.uniform(0.2, 0.9)
    rgb = rng.uniform(0, 1, 3)
    sc = one_splat_scene(cam, p, su, sv, q, o, rgb)
    # the values the oracle sees (float32 stored inputs)
    p32, q32 = sc.means[:, 0].astype(np.float64), sc.quats[:, 0].astype(np.float64)
    su32, sv32 = float(sc.scales[0, 0]), float(sc.scales[1, 0])
    o32, rgb32 = float(sc.opacity[0]), sc.rgb[:, 0].astype(np.float64)
    B = cam.F_xy[:, :3].astype(np.float64)
    b = cam.F_xy[:, 3].astype(np.float64)
    out = oracle.render(oracle.SceneF64.of(sc), cam, brute=True)
    R = rot(q32)
    vs = np.cross(B[0], B[1]); vs = vs * np.sign(vs[2]) / np.linalg.norm(vs)
    n = R[:, 2] * (1.0 if R[:, 2] @ vs >= 0 else -1.0)
    checked = 0
    for j in range(cam.height):
        for i in range(cam.width):
            a, depth, _, _ = geometric_pixel(p32, su32, sv32, q32, o32, B, b, float(cam.max_alt),
                                             i + 0.5, j + 0.5)
            if abs(a / AMIN - 1) < 1e-6:
                continue
            if a < AMIN:
                assert out["alpha"][j, i] == 0.0 and np.all(out["rgb"][:, j, i] == 0)
                continue
            checked += 1
            np.testing.assert_allclose(out["alpha"][j, i], a, rtol=1e-9, atol=1e-12)
            np.testing.assert_allclose(out["rgb"][:, j, i], a * rgb32, rtol=1e-9, atol=1e-12)
            np.testing.assert_allclose(out["depth"][j, i], a * depth, rtol=1e-9, atol=1e-12)
            np.testing.assert_allclose(out["normal"][:, j, i], a * n, rtol=1e-9, atol=1e-12)
    assert checked > 20


def test_flat_splat_nadir_closed_form():
    """Flat splat seen from nadir: r^2 = ((X - p_x)/s_u)^2 + ((Y - p_y)/s_v)^2 in a frame
    spun by the in-plane angle; depth = max_alt - p_z; normal = +z."""
    k = 20.0
    cam = H.nadir_camera(48, 48, k=k, max_alt=2.0)
    psi = 0.6
    p = np.array([0.1, -0.05, 0.3])
    su, sv, o = 0.15, 0.08, 0.7
    sc = one_splat_scene(cam, p, su, sv, H.quat_axis_angle([0, 0, 1], psi), o, [0.2, 0.5, 0.9])
    out = oracle.render(oracle.SceneF64.of(sc), cam)
    p32 = sc.means[:, 0].astype(np.float64)
    q32 = sc.quats[:, 0].astype(np.float64)
    ang = 2 * math.atan2(q32[3], q32[0])
    su32, sv32, o32 = float(sc.scales[0, 0]), float(sc.scales[1, 0]), float(sc.opacity[0])
    for (i, j) in [(24, 24), (27, 22), (20, 26), (30, 30), (25, 19)]:
        X = (i + 0.5 - 24) / k
        Y = -(j + 0.5 - 24) / k
        dx, dy = X - p32[0], Y - p32[1]
        ru = (math.cos(ang) * dx + math.sin(ang) * dy) / su32
        rv = (-math.sin(ang) * dx + math.cos(ang) * dy) / sv32
        gs = math.exp(-((i + 0.5 - (k * p32[0] + 24)) ** 2 + (j + 0.5 - (-k * p32[1] + 24)) ** 2)
                      / (2 * SIG ** 2))
        a = min(AMAX, o32 * max(math.exp(-0.5 * (ru * ru + rv * rv)), gs))
        if a < AMIN:
            continue
        assert out["alpha"][j, i] == pytest.approx(a, rel=1e-10)
        assert out["depth"][j, i] == pytest.approx(a * (float(cam.max_alt) - p32[2]), rel=1e-10)
        np.testing.assert_allclose(out["normal"][:, j, i], [0, 0, a], atol=1e-12)


def test_degenerate_edge_on_splat_uses_screen_gaussian():
    """|det M| below the threshold: only G((x - c)/sigma) remains, depth = centre depth."""
    cam = H.nadir_camera(32, 32, k=20.0, max_alt=2.0)
    # rotate the splat 90 deg about x: t_v becomes vertical, the splat is a line from above
    q = H.quat_axis_angle([1, 0, 0], math.pi / 2)
    sc = one_splat_scene(cam, [0.0, 0.0, 0.5], 0.2, 0.2, q, 0.8, [1, 1, 1])
    s64 = oracle.SceneF64.of(sc)
    pr = oracle.project(s64, cam)
    assert abs(pr["det"][0]) < OPT.det_eps and pr["deg"][0] == 1
    out = oracle.render(s64, cam)
    c = np.array([pr["cx"][0], pr["cy"][0]])
    o32 = float(sc.opacity[0])
    for (i, j) in [(16, 16), (17, 16), (15, 15), (16, 18)]:
        a = min(AMAX, o32 * math.exp(-((i + .5 - c[0]) ** 2 + (j + .5 - c[1]) ** 2) / (2 * SIG ** 2)))
        exp_a = a if a >= AMIN else 0.0
        assert out["alpha"][j, i] == pytest.approx(exp_a, rel=1e-12, abs=1e-15)
        assert out["depth"][j, i] == pytest.approx(exp_a * (2.0 - float(sc.means[2, 0])), rel=1e-12,
                                                   abs=1e-15)


def test_two_splats_composite_in_height_order():
    """Eq. rasterization with two splats: A = a1 c1 + (1 - a1) a2 c2, the higher one first,
    whatever their indices."""
    cam = H.nadir_camera(16, 16, k=10.0, max_alt=2.0)
    c_lo, c_hi = np.array([0.9, 0.1, 0.2]), np.array([0.1, 0.8, 0.3])
    # index 0 is the LOWER splat
    sc = H.make([[0.0, 0.0], [0.0, 0.0], [0.1, 0.4]], [[0.3, 0.3], [0.3, 0.3]],
                [[1, 1], [0, 0], [0, 0], [0, 0]], [0.5, 0.6], np.stack([c_lo, c_hi], 1), [cam])
    out = oracle.render(oracle.SceneF64.of(sc), cam)
    j = i = 8  # pixel centre (8.5, 8.5); splat centres at (8, 8)
    u2 = ((i + 0.5 - 8) / 10.0 / float(sc.scales[0, 0])) ** 2 + ((j + 0.5 - 8) / 10.0 / float(sc.scales[1, 0])) ** 2
    g = math.exp(-0.5 * u2)
    a_hi, a_lo = float(sc.opacity[1]) * g, float(sc.opacity[0]) * g
    rgb32 = sc.rgb.astype(np.float64)
    expect = a_hi * rgb32[:, 1] + (1 - a_hi) * a_lo * rgb32[:, 0]
    np.testing.assert_allclose(out["rgb"][:, j, i], expect, rtol=1e-12)
    assert out["alpha"][j, i] == pytest.approx(1 - (1 - a_hi) * (1 - a_lo), rel=1e-12)
    zc_hi, zc_lo = 2.0 - float(sc.means[2, 1]), 2.0 - float(sc.means[2, 0])
    assert out["depth"][j, i] == pytest.approx(a_hi * zc_hi + (1 - a_hi) * a_lo * zc_lo, rel=1e-12)


def test_equal_heights_break_ties_by_index():
    cam = H.nadir_camera(16, 16, k=10.0)
    sc = H.make([[0.0, 0.0], [0.0, 0.0], [0.2, 0.2]], [[0.3, 0.3], [0.3, 0.3]],
                [[1, 1], [0, 0], [0, 0], [0, 0]], [0.5, 0.5], [[1, 0], [0, 1], [0, 0]], [cam])
    out = oracle.render(oracle.SceneF64.of(sc), cam)
    r, g = out["rgb"][0, 8, 8], out["rgb"][1, 8, 8]
    # splat 0 (red) is in front, so it gets the larger weight
    assert r > g > 0
    assert g == pytest.approx(r * (1 - r), rel=1e-12)


def test_early_stop_excludes_the_stopping_splat():
    """T after three splats of alpha 0.95 is 1.25e-4; a fourth would take it below 1e-4,
    so it is not composited."""
    cam = H.nadir_camera(8, 8, k=10.0)
    n = 5
    heights = np.array([0.5, 0.4, 0.3, 0.2, 0.1])
    o = 0.95
    sc = H.make(np.stack([np.zeros(n), np.zeros(n), heights]), np.full((2, n), 5.0),
                np.tile([[1], [0], [0], [0]], (1, n)), np.full(n, o), np.eye(3)[:, [0, 1, 2, 0, 1]],
                [cam])
    out = oracle.render(oracle.SceneF64.of(sc), cam)
    j = i = 4
    # pixel (4.5, 4.5), centre (4, 4): u^2 = 2 * (0.05 / 5)^2
    g = math.exp(-0.5 * 2 * (0.05 / float(sc.scales[0, 0])) ** 2)
    a = float(sc.opacity[0]) * g
    T = [1.0, 1 - a, (1 - a) ** 2, (1 - a) ** 3]
    assert T[3] >= TMIN and T[3] * (1 - a) < TMIN
    assert out["ncontrib"][j, i] == 3 and out["terminated"][j, i] == 1
    assert out["alpha"][j, i] == pytest.approx(1 - T[3], rel=1e-12)
    np.testing.assert_allclose(out["rgb"][:, j, i], [a, a * T[1], a * T[2]], rtol=1e-12)


def test_alpha_clamp_and_threshold():
    cam = H.nadir_camera(16, 16, k=10.0)
    sc = one_splat_scene(cam, [0.0, 0.0, 0.1], 0.05, 0.05, [1, 0, 0, 0], 1.0, [1, 1, 1])
    out = oracle.render(oracle.SceneF64.of(sc), cam)
    # pixel (7, 7) is (0.5, 0.5) px = 0.05 units from the centre: u^2 = 2, so G(u) = e^-1,
    # while the screen-space term is exp(-0.5 / (2 sigma^2)) = e^-0.5 and wins the max
    gu = math.exp(-0.5 * 2 * (0.05 / float(sc.scales[0, 0])) ** 2)
    gs = math.exp(-0.5 / (2 * SIG ** 2))
    assert gs > gu
    assert out["alpha"][7, 7] == pytest.approx(gs, rel=1e-12)
    sc2 = one_splat_scene(cam, [0.005, -0.005, 0.1], 2.0, 2.0, [1, 0, 0, 0], 1.0, [1, 1, 1])
    out2 = oracle.render(oracle.SceneF64.of(sc2), cam)
    assert out2["alpha"][7, 8] == pytest.approx(AMAX, rel=0, abs=0)  # clamped: o G > 0.99
    # far pixels: o G < 1/255 contributes nothing
    assert out["alpha"][0, 0] == 0.0 and out["ncontrib"][0, 0] == 0


# ------------------------------------------------------------------------------ invariants
@pytest.mark.parametrize("seed", [1, 2])
def test_weights_sum_to_one_minus_T(seed):
    sc = H.random_scene(seed, n=40)
    sc.rgb[:] = 1.0
    out = oracle.render(oracle.SceneF64.of(sc), sc.cameras[0])
    for c in range(3):
        np.testing.assert_allclose(out["rgb"][c], out["alpha"], atol=1e-14)
    np.testing.assert_allclose(out["alpha"], 1 - out["T"], atol=1e-15)


def test_input_order_invariance_bitwise():
    sc = H.random_scene(3, n=60)
    perm = np.random.default_rng(0).permutation(sc.n)
    sc2 = H.make(sc.means[:, perm], sc.scales[:, perm], sc.quats[:, perm], sc.opacity[perm],
                 sc.rgb[:, perm], sc.cameras)
    assert len(np.unique(sc.means[2])) == sc.n
    a = oracle.render(oracle.SceneF64.of(sc), sc.cameras[0])
    b = oracle.render(oracle.SceneF64.of(sc2), sc.cameras[0])
    for k in ("rgb", "depth", "normal", "alpha"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("sun", [False, True])
def test_brute_equals_binned_bitwise(sun):
    sc = H.random_scene(4, n=80, width=50, height=37)
    s64 = oracle.SceneF64.of(sc)
    a = oracle.render(s64, sc.cameras[0], sun=sun, brute=True)
    b = oracle.render(s64, sc.cameras[0], sun=sun, brute=False)
    for k in ("rgb", "depth", "normal", "alpha", "T", "ncontrib"):
        assert np.array_equal(a[k], b[k]), k


def test_order_is_height_descending_then_index():
    sc = H.random_scene(5, n=50)
    sc.means[2, 10] = sc.means[2, 3]
    o = oracle.order(oracle.SceneF64.of(sc))
    z = sc.means[2].astype(np.float64)
    ref = sorted(range(sc.n), key=lambda k: (-z[k], k))
    assert list(o) == ref


def test_Q_inverts_M_and_extent_is_exact():
    sc = H.random_scene(6, n=30)
    pr = oracle.project(oracle.SceneF64.of(sc), sc.cameras[0])
    for k in range(sc.n):
        if pr["deg"][k] or pr["culled"][k]:
            continue
        M = np.array([[pr["M00"][k], pr["M01"][k]], [pr["M10"][k], pr["M11"][k]]])
        Q = np.array([[pr["Q00"][k], pr["Q01"][k]], [pr["Q10"][k], pr["Q11"][k]]])
        np.testing.assert_allclose(Q @ M, np.eye(2), atol=1e-12)
        c = np.array([pr["cx"][k], pr["cy"][k]])
        np.testing.assert_allclose(np.array([pr["q0"][k], pr["q1"][k]]), -Q @ c, rtol=1e-12)
        # support of the u term: x = c + M u, |u|^2 <= r2; its widest x reach is r |M_i,:|
        r = math.sqrt(pr["r2"][k])
        t = np.linspace(0, 2 * np.pi, 20001)
        ring = M @ np.stack([np.cos(t), np.sin(t)]) * r
        reach = np.abs(ring).max(1)
        ex = max(np.linalg.norm(M[0]), SIG) * r
        ey = max(np.linalg.norm(M[1]), SIG) * r
        assert reach[0] <= ex * (1 + 1e-12) and reach[1] <= ey * (1 + 1e-12)
        if np.linalg.norm(M[0]) > SIG:
            assert reach[0] == pytest.approx(ex, rel=1e-6)
        assert pr["ex"][k] >= ex and pr["ey"][k] >= ey


def test_colour_correction_is_C_A_plus_c():
    """Eq. image_formation, corrected albedo C A + c with a non-symmetric C."""
    sc = H.random_scene(7, n=30)
    cam = sc.cameras[0]
    rng = np.random.default_rng(1)
    col = (np.concatenate([np.eye(3), np.zeros((3, 1))], 1) + rng.normal(0, 0.3, (3, 4))).astype(np.float32)
    s64 = oracle.SceneF64.of(sc)
    a = oracle.render(s64, cam)  # identity colour
    b = oracle.render(s64, cam, color=col)
    C, c = col[:, :3].astype(np.float64), col[:, 3].astype(np.float64)
    expect = np.einsum("ij,jhw->ihw", C, a["rgb"]) + c[:, None, None]
    np.testing.assert_allclose(b["rgb"], expect, atol=1e-13)


# ------------------------------------------------------------------------------ sun camera
def test_sun_camera_nullspace_and_offset():
    """Supp. A: B_sun s = 0 for s = (cos phi / tan theta, sin phi / tan theta, 1); the sun
    view keeps the main view's offset (scaled to the shadow map)."""
    rng = np.random.default_rng(8)
    for _ in range(5):
        cam = H.oblique_camera(rng, width=40, height=40, k=25.0, off_nadir_deg=rng.uniform(0, 30))
        cam.sun_phi = float(np.float32(rng.uniform(0, 2 * np.pi)))
        cam.sun_theta = float(np.float32(rng.uniform(0.6, 1.3)))
        cam.shadow_scale = float(np.float32(0.5))
        cam.dF_xy = rng.normal(0, 0.2, (2, 4)).astype(np.float32)
        phi, th = cam.sun_phi, cam.sun_theta
        s = np.array([math.cos(phi) / math.tan(th), math.sin(phi) / math.tan(th), 1.0])
        Bs, bs, _, _ = oracle.camera(cam, sun=True)
        Bm, bm, _, _ = oracle.camera(cam, sun=False)
        np.testing.assert_allclose(Bs @ s, 0.0, atol=1e-12)
        np.testing.assert_allclose(bs, 0.5 * bm, rtol=1e-15)
        # points on the ground (z = 0) project the same up to the map scale
        p = np.array([0.3, -0.2, 0.0])
        np.testing.assert_allclose(Bs @ p + bs, 0.5 * (Bm @ p + bm), rtol=1e-12)
        # main camera = F + dF
        F = cam.F_xy.astype(np.float64) + cam.dF_xy.astype(np.float64)
        np.testing.assert_allclose(Bm, F[:, :3], rtol=1e-15)


def test_flat_ground_scene_renders_the_same_from_the_sun():
    rng = np.random.default_rng(9)
    n = 30
    cam = H.oblique_camera(rng, width=40, height=40, k=25.0, off_nadir_deg=20.0)
    cam.shadow_w = cam.shadow_h = 40
    cam.shadow_scale = 1.0
    means = np.concatenate([rng.uniform(-0.6, 0.6, (2, n)), np.zeros((1, n))], 0)
    sc = H.make(means, rng.uniform(0.05, 0.1, (2, n)), np.tile([[1], [0], [0], [0]], (1, n)),
                rng.uniform(0.1, 0.9, n), rng.uniform(0, 1, (3, n)), [cam])
    s64 = oracle.SceneF64.of(sc)
    a = oracle.render(s64, cam, sun=False)
    b = oracle.render(s64, cam, sun=True)
    np.testing.assert_allclose(a["depth"], b["depth"], atol=1e-12)
    np.testing.assert_allclose(a["alpha"], b["alpha"], atol=1e-12)


def test_translation_equivariance_of_delta_offset():
    """A delta of +1 px on b_x shifts the image one pixel to the right."""
    sc = H.random_scene(10, n=40, width=40, height=30)
    cam = sc.cameras[0]
    s64 = oracle.SceneF64.of(sc)
    a = oracle.render(s64, cam)
    dF = np.zeros((2, 4), np.float32); dF[0, 3] = 1.0
    b = oracle.render(s64, cam, dF=dF)
    for k in ("rgb", "depth", "normal", "alpha"):
        np.testing.assert_allclose(b[k][..., 1:], a[k][..., :-1], atol=1e-9)


# ------------------------------------------------------------------------------ gradients
def _tangents(rng, sc):
    return dict(means=rng.normal(size=sc.means.shape) * 0.01,
                scales=rng.normal(size=sc.scales.shape) * 0.005,
                quats=rng.normal(size=sc.quats.shape) * 0.05,
                opacity=rng.normal(size=sc.opacity.shape) * 0.05,
                rgb=rng.normal(size=sc.rgb.shape) * 0.1,
                dF=rng.normal(size=8) * np.array([0.3, 0.3, 0.3, 1.0] * 2),
                color=rng.normal(size=12) * 0.1)


def _upstream(rng, out, mask=None):
    g = dict(rgb=rng.normal(size=out["rgb"].shape), depth=rng.normal(size=out["depth"].shape),
             normal=rng.normal(size=out["normal"].shape), alpha=rng.normal(size=out["alpha"].shape),
             distort=rng.normal(size=out["distort"].shape))
    if mask is not None:
        for k in g:
            g[k] = g[k] * mask
    return g


def _dot(g, t):
    return sum(float(np.sum(g[k] * t[k])) for k in g)


def _adjoint_dot(grads, tang):
    s = 0.0
    for k in ("means", "scales", "quats", "opacity", "rgb"):
        s += float(np.sum(grads[k] * tang[k]))
    s += float(np.sum(grads["dF"].ravel() * tang["dF"]))
    s += float(np.sum(grads["color"].ravel() * tang["color"]))
    return s


@pytest.mark.parametrize("seed,sun", [(11, False), (12, False), (13, True), (14, True)])
def test_adjoint_equals_dual_numbers(seed, sun):
    sc = H.random_scene(seed, n=30, width=32, height=24, delta=True, color_noise=0.05)
    cam = sc.cameras[0]
    s64 = oracle.SceneF64.of(sc)
    rng = np.random.default_rng(seed)
    out = oracle.render(s64, cam, sun=sun)
    g = _upstream(rng, out)
    if sun:
        g["rgb"] = None; g["normal"] = None
    tang = _tangents(rng, sc)
    if sun:
        tang["color"] = np.zeros(12)
    d = oracle.render_dual(s64, cam, tang, sun=sun)
    lhs = sum(float(np.sum(g[k] * d[k])) for k in g if g[k] is not None)
    grads = oracle.backward(s64, cam, g, sun=sun)
    rhs = _adjoint_dot(grads, tang)
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


@pytest.mark.parametrize("seed,sun", [(21, False), (22, True)])
def test_adjoint_equals_central_differences(seed, sun):
    sc = H.random_scene(seed, n=16, width=24, height=20, delta=True, color_noise=0.05)
    cam = sc.cameras[0]
    s64 = oracle.SceneF64.of(sc)
    rng = np.random.default_rng(seed)
    out = oracle.render(s64, cam, sun=sun)
    mask = (out["margin_bwd"] > 1e-3).astype(np.float64)
    g = _upstream(rng, out, mask)
    if sun:
        g["rgb"] = None; g["normal"] = None
    tang = _tangents(rng, sc)
    if sun:
        tang["color"] = np.zeros(12)
    grads = oracle.backward(s64, cam, g, sun=sun)
    rhs = _adjoint_dot(grads, tang)

    def f(h):
        s2 = oracle.SceneF64(s64.means + h * tang["means"], s64.scales + h * tang["scales"],
                             s64.quats + h * tang["quats"], s64.opacity + h * tang["opacity"],
                             s64.rgb + h * tang["rgb"])
        rec_dF = cam.dF_xy.astype(np.float64).ravel() + h * tang["dF"]
        col = cam.color.astype(np.float64).ravel() + h * tang["color"]
        o = _render_f64(s2, cam, sun, rec_dF, col)
        return sum(float(np.sum(g[k] * o[k])) for k in g if g[k] is not None)

    h = 1e-6
    fd = (f(h) - f(-h)) / (2 * h)
    assert abs(fd - rhs) <= 1e-6 * max(1.0, abs(rhs)), (fd, rhs)


def _render_f64(s64, cam, sun, dF_flat, col_flat):
    """Render with float64 camera delta / colour (no float32 rounding), for differences."""
    import ctypes
    rec = oracle.camera_record(cam)
    rec[oracle.C_DF:oracle.C_DF + 8] = dF_flat
    rec[oracle.C_COLOR:oracle.C_COLOR + 12] = col_flat
    W, H_ = (cam.shadow_w, cam.shadow_h) if sun else (cam.width, cam.height)
    o = oracle.Opts().record()
    out = dict(rgb=np.zeros((3, H_, W)), depth=np.zeros((H_, W)), normal=np.zeros((3, H_, W)),
               alpha=np.zeros((H_, W)), distort=np.zeros((H_, W)))
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    col = np.ascontiguousarray(col_flat)
    oracle.lib().ora_render(*s64.args(), P(rec), int(sun), P(col), P(o), 0, 0, W, H_, 0,
                            P(out["rgb"]), P(out["depth"]), P(out["normal"]), P(out["alpha"]),
                            None, None, None, None, None, P(out["distort"]))
    return out


def test_grad_dF_equals_grad_F():
    """F' = F + dF: the gradient with respect to the delta is the gradient with respect to F."""
    sc = H.random_scene(31, n=20, width=24, height=20, delta=True)
    cam = sc.cameras[0]
    s64 = oracle.SceneF64.of(sc)
    rng = np.random.default_rng(3)
    out = oracle.render(s64, cam)
    g = _upstream(rng, out, (out["margin_bwd"] > 1e-3).astype(float))
    grads = oracle.backward(s64, cam, g)
    for idx in [(0, 0), (1, 2), (0, 3), (1, 3)]:
        h = 1e-5
        fvals = []
        for sgn in (1, -1):
            c2 = H.nadir_camera()
            c2.__dict__.update(cam.__dict__)
            F = cam.F_xy.astype(np.float64).copy()
            F[idx] += sgn * h
            rec = oracle.camera_record(cam)
            rec[oracle.C_F:oracle.C_F + 8] = F.ravel()
            import ctypes
            P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
            o = oracle.Opts().record()
            col = rec[oracle.C_COLOR:oracle.C_COLOR + 12].copy()
            pl = dict(rgb=np.zeros((3, cam.height, cam.width)), depth=np.zeros((cam.height, cam.width)),
                      normal=np.zeros((3, cam.height, cam.width)), alpha=np.zeros((cam.height, cam.width)),
                      distort=np.zeros((cam.height, cam.width)))
            oracle.lib().ora_render(*s64.args(), P(rec), 0, P(col), P(o), 0, 0, cam.width, cam.height,
                                    0, P(pl["rgb"]), P(pl["depth"]), P(pl["normal"]), P(pl["alpha"]),
                                    None, None, None, None, None, P(pl["distort"]))
            fvals.append(sum(float(np.sum(g[k] * pl[k])) for k in g))
        fd = (fvals[0] - fvals[1]) / (2 * h)
        assert fd == pytest.approx(grads["dF"][idx], rel=1e-5, abs=1e-6)


def test_normal_is_flipped_to_face_the_sensor():
    """The normal output is R[:, 2] oriented toward the camera: an upside-down splat
    (rotated by pi about x) still reports an upward normal under a nadir view, and under
    an oblique view the reported normal has a non-negative dot product with the view axis."""
    cam = H.nadir_camera(16, 16, k=10.0)
    q = H.quat_axis_angle([1, 0, 0], math.pi * 0.999)
    sc = one_splat_scene(cam, [0.0, 0.0, 0.1], 0.3, 0.3, q, 0.5, [1, 1, 1])
    out = oracle.render(oracle.SceneF64.of(sc), cam)
    a = out["alpha"][8, 8]
    R = rot(sc.quats[:, 0].astype(np.float64))
    assert R[2, 2] < 0
    np.testing.assert_allclose(out["normal"][:, 8, 8], -a * R[:, 2], rtol=1e-12)
    rng = np.random.default_rng(44)
    for _ in range(4):
        cam = H.oblique_camera(rng, width=24, height=24, k=10.0, off_nadir_deg=rng.uniform(10, 40))
        qq = H.quat_axis_angle(rng.normal(size=3), rng.uniform(1.7, 3.0))
        sc = one_splat_scene(cam, [0.0, 0.0, 0.0], 0.4, 0.4, qq, 0.5, [1, 1, 1])
        B = cam.F_xy[:, :3].astype(np.float64)
        vs = np.cross(B[0], B[1]); vs *= np.sign(vs[2])
        R = rot(sc.quats[:, 0].astype(np.float64))
        out = oracle.render(oracle.SceneF64.of(sc), cam)
        nn = out["normal"][:, 12, 12]
        assert out["alpha"][12, 12] > 0
        np.testing.assert_allclose(np.abs(nn), out["alpha"][12, 12] * np.abs(R[:, 2]), rtol=1e-12)
        assert nn @ vs >= 0
