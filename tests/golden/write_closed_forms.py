"""Writes closed_forms.json: rendered values that follow from the paper's equations by hand,
for scenes of one to five splats under a nadir affine camera (x = k X + W/2, y = -k Y + H/2),
computed here with `math` alone (no oracle, no rasterizer).

Each case states the passage it follows and its derivation.  Inputs are rounded to float32
first (both implementations read float32 values); the closed forms are then evaluated in
float64.  The rasterizer constants are the float32 values of sigma = 1/sqrt(2) px (the
screen-space low-pass of the lower-bounded Gaussian, Sec. 3.2), alpha_min = 1/255,
alpha_max = 0.99 and T_min = 1e-4.

Run from the repository root:  python -m tests.golden.write_closed_forms
"""
from __future__ import annotations

import math

import numpy as np

import scenegen
from tests.golden import fixtures as FX

F = lambda x: float(np.float32(x))
SIG = F(1.0 / math.sqrt(2.0))
AMIN, AMAX, TMIN = F(1.0 / 255.0), F(0.99), F(1e-4)


def nadir(width, height, k, max_alt=2.0, color=None, phi=0.3, theta=0.9, shadow=None):
    Fxy = np.array([[k, 0.0, 0.0, width / 2.0], [0.0, -k, 0.0, height / 2.0]], np.float32)
    col = np.concatenate([np.eye(3), np.zeros((3, 1))], 1) if color is None else np.asarray(color)
    sw, sh = (width, height) if shadow is None else shadow
    return scenegen.Camera(F_xy=Fxy, dF_xy=np.zeros((2, 4), np.float32), max_alt=F(max_alt),
                           width=width, height=height, color=col.astype(np.float32), sun_phi=F(phi),
                           sun_theta=F(theta), shadow_w=sw, shadow_h=sh, shadow_scale=1.0)


def quat_z(psi):
    return [math.cos(psi / 2), 0.0, 0.0, math.sin(psi / 2)]


def alpha_of(o, gu, gs):
    """Lower-bounded Gaussian, clamp and threshold (Sec. 3.2): o max(G(u), G((x - c)/sigma))."""
    raw = o * max(gu, gs)
    # keep clear of the two decisions, so that float32 and float64 evaluations take them alike
    assert abs(raw - AMIN) > 1e-6 and abs(raw - AMAX) > 1e-6
    a = min(AMAX, raw)
    return a if a >= AMIN else 0.0


def flat_splat(k, cx, cy, psi, su, sv, px, py):
    """A splat lying in a horizontal plane, rotated by psi about z, seen from nadir: the pixel
    centre (px, py) is the world offset (dX, dY) = ((px - cx)/k, -(py - cy)/k) from the centre,
    u = (dX cos psi + dY sin psi)/s_u, v = (-dX sin psi + dY cos psi)/s_v (Eq. affine2dgs_screen2uv
    solved by hand).  Returns u, v, G(u), G((x - c)/sigma) and dX, dY."""
    dX, dY = (px - cx) / k, -(py - cy) / k
    u = (math.cos(psi) * dX + math.sin(psi) * dY) / su
    v = (-math.sin(psi) * dX + math.cos(psi) * dY) / sv
    gu = math.exp(-0.5 * (u * u + v * v))
    gs = math.exp(-((px - cx) ** 2 + (py - cy) ** 2) / (2.0 * SIG * SIG))
    return u, v, gu, gs, dX, dY


def case_flat_rotated():
    k, W, H = 20.0, 48, 48
    cam = nadir(W, H, k)
    p = [F(0.1), F(-0.05), F(0.3)]
    q = [F(x) for x in quat_z(0.6)]
    psi = 2.0 * math.atan2(q[3], q[0])  # the float32 quaternion's angle (normalisation keeps it)
    su, sv, o = F(0.15), F(0.08), F(0.7)
    rgb = [F(0.2), F(0.5), F(0.9)]
    cx, cy = k * p[0] + W / 2, -k * p[1] + H / 2
    pixels, exp = [], dict(alpha=[], depth=[], rgb=[], normal=[])
    for (i, j) in [(24, 24), (27, 22), (20, 26), (30, 30), (25, 19), (15, 24), (26, 16)]:
        _, _, gu, gs, _, _ = flat_splat(k, cx, cy, psi, su, sv, i + 0.5, j + 0.5)
        a = alpha_of(o, gu, gs)
        pixels.append([i, j])
        exp["alpha"].append(a)
        exp["depth"].append(a * (cam.max_alt - p[2]))  # Eq. depth_affine_camera: b_z - p_z
        exp["rgb"].append([a * c for c in rgb])
        exp["normal"].append([0.0, 0.0, a])  # R[:, 2] = +z faces the nadir sensor
    # gradient of L = alpha + g . rgb_out at pixel P: L = alpha (1 + g . rgb)
    P, g = (27, 22), [0.3, -0.2, 0.5]
    u, v, gu, gs, dX, dY = flat_splat(k, cx, cy, psi, su, sv, P[0] + 0.5, P[1] + 0.5)
    a = alpha_of(o, gu, gs)
    assert gu > gs and AMIN <= a < AMAX  # the object-space Gaussian decides, no clamp
    m = 1.0 + sum(gc * c for gc, c in zip(g, rgb))
    c, s = math.cos(psi), math.sin(psi)
    # E = -(u^2 + v^2)/2 with du/dp_x = -cos/s_u, dv/dp_x = sin/s_v, du/dp_y = -sin/s_u,
    # dv/dp_y = -cos/s_v, du/ds_u = -u/s_u, dv/ds_v = -v/s_v; d alpha = alpha dE
    dEx = u * c / su - v * s / sv
    dEy = u * s / su + v * c / sv
    grad = dict(means=[m * a * dEx, m * a * dEy, 0.0], scales=[m * a * u * u / su, m * a * v * v / sv],
                opacity=[m * a / o], rgb=[a * gc for gc in g])
    return dict(name="flat_rotated_anisotropic", view="main",
                cite="Sec. 3.1 Eq. 2dgs_splat_param; Sec. 3.2 Eq. affine2dgs_screen2uv, Eq. affine2dgs_Qq, "
                     "Eq. depth_affine_camera, the lower-bounded Gaussian",
                derivation="one horizontal splat rotated by psi about z under a nadir camera: "
                           "u, v from the world offset of the pixel centre in the splat frame; "
                           "alpha = min(0.99, o max(exp(-(u^2+v^2)/2), exp(-|x-c|^2/(2 sigma^2)))), "
                           "zero below 1/255; depth = alpha (b_z - p_z); normal = alpha e_z; "
                           "rgb = alpha rgb.  Gradient of alpha + g . rgb_out at one pixel: "
                           "(1 + g . rgb) alpha dE, dE from E = -(u^2 + v^2)/2 (quaternion "
                           "gradients not stated)",
                splats=FX.splats_json(p, [su, sv], q, [o], rgb), camera=FX.camera_json(cam),
                pixels=pixels, expected=exp,
                grad=dict(pixel=list(P), d_alpha=1.0, d_rgb=g, expected=grad))


def case_two_splats():
    k, W, H = 10.0, 16, 16
    cam = nadir(W, H, k)
    c_lo, c_hi = [F(0.9), F(0.1), F(0.2)], [F(0.1), F(0.8), F(0.3)]
    h_lo, h_hi = F(0.1), F(0.4)
    s, o_lo, o_hi = F(0.3), F(0.5), F(0.6)
    pixels, exp = [], dict(alpha=[], depth=[], rgb=[])
    for (i, j) in [(8, 8), (9, 7), (6, 10)]:
        _, _, gu, gs, _, _ = flat_splat(k, 8.0, 8.0, 0.0, s, s, i + 0.5, j + 0.5)
        a_hi, a_lo = alpha_of(o_hi, gu, gs), alpha_of(o_lo, gu, gs)
        # Eq. rasterization, higher splat first: f = a1 f1 + (1 - a1) a2 f2
        pixels.append([i, j])
        exp["alpha"].append(1.0 - (1.0 - a_hi) * (1.0 - a_lo))
        exp["depth"].append(a_hi * (cam.max_alt - h_hi) + (1 - a_hi) * a_lo * (cam.max_alt - h_lo))
        exp["rgb"].append([a_hi * x + (1 - a_hi) * a_lo * y for x, y in zip(c_hi, c_lo)])
    # index 0 is the lower splat: the order comes from the heights, not the indices
    return dict(name="two_splats_height_order", view="main",
                cite="Sec. 3.2 Eq. rasterization and the height-based sort",
                derivation="two concentric horizontal splats; the higher (index 1) composites "
                           "first: alpha = 1 - (1 - a_hi)(1 - a_lo), f = a_hi f_hi + (1 - a_hi) a_lo f_lo",
                splats=FX.splats_json([[0.0, 0.0], [0.0, 0.0], [h_lo, h_hi]], [[s, s], [s, s]],
                                      [[1, 1], [0, 0], [0, 0], [0, 0]], [o_lo, o_hi],
                                      np.stack([c_lo, c_hi], 1)),
                camera=FX.camera_json(cam), pixels=pixels, expected=exp)


def case_early_stop():
    k, W, H, n = 10.0, 8, 8, 5
    cam = nadir(W, H, k)
    hs = [F(x) for x in (0.5, 0.4, 0.3, 0.2, 0.1)]
    s, o = F(5.0), F(0.95)
    cols = np.eye(3)[:, [0, 1, 2, 0, 1]]
    i = j = 4
    _, _, gu, gs, _, _ = flat_splat(k, 4.0, 4.0, 0.0, s, s, i + 0.5, j + 0.5)
    a = alpha_of(o, gu, gs)
    T = [1.0]
    for _ in range(4):
        T.append(T[-1] * (1.0 - a))
    # three splats leave T = (1 - a)^3 >= T_min; the fourth would take it below: not composited
    assert T[3] >= TMIN > T[4]
    rgb = [sum(a * T[m] * cols[c, m] for m in range(3)) for c in range(3)]
    depth = sum(a * T[m] * (cam.max_alt - hs[m]) for m in range(3))
    return dict(name="early_stop", view="main",
                cite="Sec. 3.2 Eq. rasterization, front-to-back blending with early termination",
                derivation="five concentric wide splats of alpha about 0.95: after three, T = (1 - a)^3 "
                           "= 1.25e-4 >= 1e-4 and a fourth would take T below 1e-4, so only three "
                           "are composited (the stopping splat is excluded)",
                splats=FX.splats_json(np.stack([np.zeros(n), np.zeros(n), hs]), np.full((2, n), s),
                                      np.tile([[1], [0], [0], [0]], (1, n)), np.full(n, o), cols),
                camera=FX.camera_json(cam), pixels=[[i, j]],
                expected=dict(alpha=[1.0 - T[3]], depth=[depth], rgb=[rgb]))


def case_sun_view():
    k, W, H = 20.0, 40, 32
    phi, theta = F(0.4), F(0.9)
    cam = nadir(W, H, k, phi=phi, theta=theta)
    p = [F(0.05), F(-0.1), F(0.25)]
    su, sv, o = F(0.1), F(0.07), F(0.8)
    # B_sun = B'(I - s e_z^T), s = (cos phi / tan theta, sin phi / tan theta, 1): the centre
    # moves by -p_z (s_x, s_y) on the ground before the nadir projection (Supp. A)
    sx, sy = math.cos(phi) / math.tan(theta), math.sin(phi) / math.tan(theta)
    cx, cy = k * (p[0] - p[2] * sx) + W / 2, -k * (p[1] - p[2] * sy) + H / 2
    pixels, exp = [], dict(alpha=[], depth=[])
    ci, cj = int(math.floor(cx)), int(math.floor(cy))
    for (i, j) in [(ci, cj), (ci + 1, cj), (ci - 2, cj + 1), (ci + 2, cj - 3), (ci + 1, cj + 2)]:
        _, _, gu, gs, _, _ = flat_splat(k, cx, cy, 0.0, su, sv, i + 0.5, j + 0.5)
        a = alpha_of(o, gu, gs)
        pixels.append([i, j])
        exp["alpha"].append(a)
        exp["depth"].append(a * (cam.max_alt - p[2]))  # the sun depth keeps the elevation (Sec. 3.3)
    return dict(name="sun_view_displacement", view="sun",
                cite="Sec. 3.3 Eq. sun_camera_Bxy; Supp. A (flattening along the sun direction)",
                derivation="a horizontal splat at height p_z seen from the sun: its footprint keeps "
                           "the nadir shape (t_u, t_v have no z component) and is centred at "
                           "B'(p - p_z s) + b'; alpha as for the main view; depth = alpha (b_z - p_z)",
                splats=FX.splats_json(p, [su, sv], [1, 0, 0, 0], [o], [1, 1, 1]),
                camera=FX.camera_json(cam), pixels=pixels, expected=exp)


def case_colour_correction():
    k, W, H = 20.0, 24, 20
    C = [[0.9, 0.1, 0.05, 0.01], [0.02, 1.1, -0.03, -0.02], [0.04, 0.06, 0.8, 0.03]]
    cam = nadir(W, H, k, color=C)
    C32 = np.asarray(C, np.float32).astype(np.float64)
    p = [F(0.0), F(0.0), F(0.2)]
    s, o = F(0.12), F(0.6)
    rgb = np.array([F(0.7), F(0.3), F(0.5)])
    pixels, exp = [], dict(rgb=[], alpha=[])
    for (i, j) in [(12, 10), (13, 9), (2, 2)]:  # the last pixel sees no splat: rgb = c
        _, _, gu, gs, _, _ = flat_splat(k, 12.0, 10.0, 0.0, s, s, i + 0.5, j + 0.5)
        a = alpha_of(o, gu, gs)
        pixels.append([i, j])
        exp["alpha"].append(a)
        exp["rgb"].append((C32[:, :3] @ (a * rgb) + C32[:, 3]).tolist())
    return dict(name="colour_correction", view="main",
                cite="Sec. 3.1 Eq. image_formation, the corrected albedo C A + c",
                derivation="one splat, non-symmetric C and offset c: rgb_out = C (alpha rgb) + c; "
                           "a pixel that no splat covers shows c",
                splats=FX.splats_json(p, [s, s], [1, 0, 0, 0], [o], rgb), camera=FX.camera_json(cam),
                pixels=pixels, expected=exp)


def case_edge_on():
    k, W, H = 10.0, 32, 32
    cam = nadir(W, H, k)
    w = F(math.cos(math.pi / 4))
    # 90 degrees about x: R[1][1] = (w^2 - x^2)/(w^2 + x^2) vanishes to rounding, and with
    # k^2 s_u s_v = 0.25 px^2 the determinant stays far below the 1e-6 px^2 threshold in float32 too
    q = [w, w, 0.0, 0.0]
    p = [F(0.0), F(0.0), F(0.5)]
    su, sv, o = F(0.05), F(0.05), F(0.8)
    cx, cy = 16.0, 16.0
    pixels, exp = [], dict(alpha=[], depth=[])
    for (i, j) in [(16, 16), (17, 16), (15, 15), (16, 18), (14, 17)]:
        gs = math.exp(-((i + 0.5 - cx) ** 2 + (j + 0.5 - cy) ** 2) / (2.0 * SIG * SIG))
        a = alpha_of(o, 0.0, gs)
        pixels.append([i, j])
        exp["alpha"].append(a)
        exp["depth"].append(a * (cam.max_alt - p[2]))
    return dict(name="edge_on_degenerate", view="main",
                cite="Sec. 3.2, the degenerate (edge-on) case of the lower-bounded Gaussian",
                derivation="a splat seen edge-on has |det(B R S')| far below the threshold: only the screen-space "
                           "term G((x - c)/sigma) remains and the depth is the centre's, b_z - p_z",
                splats=FX.splats_json(p, [su, sv], q, [o], [1, 1, 1]), camera=FX.camera_json(cam),
                pixels=pixels, expected=exp)


def _rounded(case: dict) -> dict:
    case["expected"] = {k: FX.g12(v) for k, v in case["expected"].items()}
    if "grad" in case:
        case["grad"]["expected"] = {k: FX.g12(v) for k, v in case["grad"]["expected"].items()}
    return case


def build() -> dict:
    return dict(
        description="Rendered values of tiny scenes that follow from the paper's equations by hand "
                    "(float64 closed forms of float32 inputs); pixel (i, j) is column i, row j; "
                    "expected values are the unnormalised planes: rgb after colour correction, "
                    "depth and normal blended with the weights, alpha = 1 - T",
        writer="tests/golden/write_closed_forms.py",
        cases=[_rounded(c()) for c in (case_flat_rotated, case_two_splats, case_early_stop, case_sun_view,
                                       case_colour_correction, case_edge_on)])


if __name__ == "__main__":
    FX.dump(build(), "closed_forms.json")
