"""FP64 CPU oracle of the sun-visibility shading and the full image formation.

TEST INFRASTRUCTURE ONLY: like the rest of ``oracle/``, only the test-suite may import it.  It
shares no code with the CUDA path.  Plain numpy in float64, vectorised over the pixels of one
view, with the adjoint written out by hand.

What it computes (per main-view pixel x = (i + 0.5, j + 0.5)):

  image formation, Sec. 3.1 Eq. image_formation:
      I = (C A + c) * (V + (1 - V) L_a)            (element-wise over the 3 channels)
  where C A + c is the rasterizer's corrected albedo and L_a the view's ambient light;

  sun visibility V, Sec. 3.1 (shadow map softened by exponential shadow mapping, as in the work
  the paper follows) and Sec. 3.3 (sun camera, depth along the sun direction kept as the
  original elevation):
      z   = D / alpha                 receiver depth (alpha-normalised rendered depth)
      h   = max_alt - z               its height (depth row B_z = [0, 0, -1], b_z = max_alt)
      u   = S (x - h B' s)            where the sun ray through the receiver meets the sun view:
                                      the sun camera flattens a point P along s onto z = 0 and
                                      projects it with S B' (Eq. sun_camera_Bxy, Supp. A), and
                                      B' P + b' = x, so S (B' (P - h s) + b') = S (x - h B' s)
      z_o = bilinear sample of D_sun / alpha_sun at u (texel centres at +0.5)
      V   = exp(-k max(z - z_o - bias, 0))      (1 when lit, smaller the deeper in shadow)
  A pixel without a surface (alpha < eps), or whose sample needs a texel outside the sun view or
  without a surface, is lit (V = 1).  k, bias and eps are readings (the paper takes the filter
  from earlier work without stating its constants); they come in as arguments.
"""
from __future__ import annotations

import numpy as np


def sun_direction(phi: float, theta: float) -> np.ndarray:
    """s = (cos phi / tan theta, sin phi / tan theta, 1) (Sec. 3.3, Supp. A)."""
    phi, theta = float(np.float32(phi)), float(np.float32(theta))
    return np.array([np.cos(phi) / np.tan(theta), np.sin(phi) / np.tan(theta), 1.0])


def camera_Bp(cam, dF=None) -> np.ndarray:
    """B' = (F + dF)[:, :3] of a view: the camera's float32 values widened exactly; an explicit
    dF is taken as given (float64)."""
    F = np.asarray(cam.F_xy, np.float32).astype(np.float64)
    d = np.asarray(cam.dF_xy, np.float32).astype(np.float64) if dF is None else np.asarray(dF, np.float64)
    return (F + d)[:, :3]


def _geometry(depth, alpha, sun_depth, sun_alpha, cam, dF, eps):
    H, W = depth.shape
    Hs, Ws = sun_depth.shape
    Bs = camera_Bp(cam, dF) @ sun_direction(cam.sun_phi, cam.sun_theta)
    S = float(np.float32(cam.shadow_scale))
    maxalt = float(np.float32(cam.max_alt))
    y, x = np.mgrid[0:H, 0:W].astype(np.float64) + 0.5
    surf = alpha >= eps
    z = np.where(surf, depth / np.where(surf, alpha, 1.0), 0.0)
    h = maxalt - z
    ux = S * (x - h * Bs[0])
    uy = S * (y - h * Bs[1])
    tx, ty = ux - 0.5, uy - 0.5
    i0, j0 = np.floor(tx).astype(np.int64), np.floor(ty).astype(np.int64)
    fx, fy = tx - i0, ty - j0
    inside = (i0 >= 0) & (i0 + 1 < Ws) & (j0 >= 0) & (j0 + 1 < Hs)
    ic, jc = np.clip(i0, 0, Ws - 2), np.clip(j0, 0, Hs - 2)
    ssurf = sun_alpha >= eps
    zs = np.where(ssurf, sun_depth / np.where(ssurf, sun_alpha, 1.0), 0.0)
    taps = [(0, 0), (1, 0), (0, 1), (1, 1)]
    tap_ok = np.ones_like(surf)
    for di, dj in taps:
        tap_ok &= ssurf[jc + dj, ic + di]
    valid = surf & inside & tap_ok
    w = [(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy]
    zo = sum(wk * zs[jc + dj, ic + di] for wk, (di, dj) in zip(w, taps))
    return dict(z=z, h=h, ux=ux, uy=uy, fx=fx, fy=fy, ic=ic, jc=jc, zs=zs, zo=zo, valid=valid, Bs=Bs, S=S,
                taps=taps, w=w)


def sun_position(depth, alpha, cam, eps, dF=None):
    """u = S (x - h B' s): where the sun ray through each main-view pixel's receiver meets the
    sun view (pixel coordinates, texel centres at +0.5)."""
    dummy = np.ones((2, 2))
    g = _geometry(depth, alpha, dummy, dummy, cam, dF, eps)
    return g["ux"], g["uy"]


def shade_forward(rgb, depth, alpha, sun_depth, sun_alpha, cam, La, k, bias, eps, dF=None):
    """I (3, H, W) and V (H, W) of one view from its rasterized planes (float64 arrays)."""
    g = _geometry(depth, alpha, sun_depth, sun_alpha, cam, dF, eps)
    delta = g["z"] - g["zo"] - bias
    V = np.where(g["valid"] & (delta > 0), np.exp(-k * np.maximum(delta, 0.0)), 1.0)
    La = np.asarray(La, np.float64)[:, None, None]
    I = rgb * (La + V * (1.0 - La))
    return I, V


def shade_backward(d_image, rgb, depth, alpha, sun_depth, sun_alpha, cam, La, k, bias, eps, dF=None):
    """Reverse-mode adjoint of shade_forward for the upstream gradient d_image (3, H, W).
    Returns d_rgb, d_depth, d_alpha, d_sun_depth, d_sun_alpha, d_La (3) and d_dF (2, 4)."""
    g = _geometry(depth, alpha, sun_depth, sun_alpha, cam, dF, eps)
    delta = g["z"] - g["zo"] - bias
    shadowed = g["valid"] & (delta > 0)
    V = np.where(shadowed, np.exp(-k * np.maximum(delta, 0.0)), 1.0)
    La = np.asarray(La, np.float64)
    shading = La[:, None, None] + V * (1.0 - La[:, None, None])
    d_rgb = d_image * shading
    dV = np.sum(d_image * rgb * (1.0 - La[:, None, None]), axis=0)
    d_La = np.sum(d_image * rgb * (1.0 - V), axis=(1, 2))
    # V = exp(-k delta) on shadowed pixels, delta = z - z_o - bias
    d_delta = np.where(shadowed, -k * V * dV, 0.0)
    dz = d_delta.copy()
    dzo = -d_delta
    # z_o = sum_t w_t zs_t: taps and the sample position u
    zs, ic, jc, fx, fy = g["zs"], g["ic"], g["jc"], g["fx"], g["fy"]
    z00, z10 = zs[jc, ic], zs[jc, ic + 1]
    z01, z11 = zs[jc + 1, ic], zs[jc + 1, ic + 1]
    dzo_dux = (1 - fy) * (z10 - z00) + fy * (z11 - z01)
    dzo_duy = (1 - fx) * (z01 - z00) + fx * (z11 - z10)
    dux, duy = dzo * dzo_dux, dzo * dzo_duy
    d_zs = np.zeros_like(zs)
    for wk, (di, dj) in zip(g["w"], g["taps"]):
        np.add.at(d_zs, (jc + dj, ic + di), np.where(shadowed, wk * dzo, 0.0))
    # u = S (x - h B' s): du/dh = -S B' s, du/dB'_ij = -S h s_j
    S, Bs, h = g["S"], g["Bs"], g["h"]
    dh = -S * (dux * Bs[0] + duy * Bs[1])
    s = sun_direction(cam.sun_phi, cam.sun_theta)
    d_dF = np.zeros((2, 4))
    for j in range(3):
        d_dF[0, j] = np.sum(-S * h * s[j] * dux)
        d_dF[1, j] = np.sum(-S * h * s[j] * duy)
    # h = max_alt - z; z = D / alpha
    dz = dz - dh
    surf = alpha >= eps
    a_safe = np.where(surf, alpha, 1.0)
    d_depth = np.where(surf, dz / a_safe, 0.0)
    d_alpha = np.where(surf, -dz * depth / (a_safe * a_safe), 0.0)
    ssurf = sun_alpha >= eps
    sa = np.where(ssurf, sun_alpha, 1.0)
    d_sun_depth = np.where(ssurf, d_zs / sa, 0.0)
    d_sun_alpha = np.where(ssurf, -d_zs * sun_depth / (sa * sa), 0.0)
    return dict(rgb=d_rgb, depth=d_depth, alpha=d_alpha, sun_depth=d_sun_depth, sun_alpha=d_sun_alpha,
                La=d_La, dF=d_dF)


def shade_margin(depth, alpha, sun_depth, sun_alpha, cam, k, bias, eps, dF=None):
    """Per pixel, the distance of the decisions to their thresholds, for excluding the pixels
    where FP32 may decide differently: receiver alpha vs eps, sample texels vs the sun view's
    edge and vs eps, and delta vs 0 (scaled by k).  Larger is safer."""
    g = _geometry(depth, alpha, sun_depth, sun_alpha, cam, dF, eps)
    m = np.abs(alpha - eps) / max(eps, 1e-30)
    frac = np.minimum(np.minimum(g["fx"], 1 - g["fx"]), np.minimum(g["fy"], 1 - g["fy"]))
    Hs, Ws = sun_depth.shape
    tx = g["ic"] + g["fx"]
    ty = g["jc"] + g["fy"]
    edge = np.minimum(np.minimum(tx, Ws - 1 - tx), np.minimum(ty, Hs - 1 - ty))
    m = np.minimum(m, np.where(np.abs(edge) < 1.0, np.abs(edge), 1.0))
    sa = np.abs(sun_alpha - eps) / max(eps, 1e-30)
    near = np.ones_like(m)
    for di, dj in g["taps"]:
        near = np.minimum(near, sa[g["jc"] + dj, g["ic"] + di])
    m = np.minimum(m, near)
    delta = g["z"] - g["zo"] - bias
    m = np.minimum(m, np.abs(delta) * k)
    return m, frac
