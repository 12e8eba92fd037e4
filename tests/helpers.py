"""Hand-built scenes and cameras for the tests (no rasterizer arithmetic here)."""
import math

import numpy as np

import scenegen


def nadir_camera(width=64, height=64, k=20.0, max_alt=2.0, color=None, dF=None,
                 sun_phi=0.3, sun_theta=0.9, shadow_scale=1.0):
    """Camera looking straight down: x = k * X + W/2, y = -k * Y + H/2 (pixels)."""
    F = np.array([[k, 0.0, 0.0, width / 2.0], [0.0, -k, 0.0, height / 2.0]], dtype=np.float32)
    col = np.concatenate([np.eye(3), np.zeros((3, 1))], 1) if color is None else color
    return scenegen.Camera(F_xy=F, dF_xy=np.zeros((2, 4), np.float32) if dF is None else
                           np.asarray(dF, np.float32), max_alt=float(np.float32(max_alt)),
                           width=width, height=height, color=np.asarray(col, np.float32),
                           sun_phi=float(np.float32(sun_phi)), sun_theta=float(np.float32(sun_theta)),
                           shadow_w=int(round(width * shadow_scale)),
                           shadow_h=int(round(height * shadow_scale)),
                           shadow_scale=float(np.float32(shadow_scale)))


def oblique_camera(rng, width=64, height=48, k=20.0, off_nadir_deg=25.0, max_alt=2.0):
    cam = scenegen.make_camera(rng, width=width, height=height, scale_m=1.0,
                               off_nadir_deg=off_nadir_deg, target_m=(0.0, 0.0, 0.0))
    # make_camera uses pixels-per-world-unit = scale_m / GSD; rescale to k
    F = cam.F_xy.astype(np.float64)
    B = F[:, :3] * (k / (1.0 / scenegen.GSD_M))
    b = np.array([width / 2.0, height / 2.0])
    cam.F_xy = np.concatenate([B, b[:, None]], 1).astype(np.float32)
    cam.max_alt = float(np.float32(max_alt))
    cam.dF_xy = np.zeros((2, 4), np.float32)
    return cam


def quat_axis_angle(axis, angle):
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    return np.concatenate([[math.cos(angle / 2)], axis * math.sin(angle / 2)])


def make(means, scales, quats, opacity, rgb, cams, scale_m=1.0):
    return scenegen.Scene(means=np.asarray(means, np.float32).reshape(3, -1),
                          scales=np.asarray(scales, np.float32).reshape(2, -1),
                          quats=np.asarray(quats, np.float32).reshape(4, -1),
                          opacity=np.asarray(opacity, np.float32).reshape(-1),
                          rgb=np.asarray(rgb, np.float32).reshape(3, -1),
                          cameras=list(cams), scale_m=scale_m)


def random_scene(seed, n=24, width=40, height=32, extent=1.0, k=30.0, oblique=True, cap=30.0,
                 scale_range=(0.03, 0.12), delta=False, color_noise=0.0):
    """A tiny random scene in world units (x, y in [-extent/2, extent/2])."""
    rng = np.random.default_rng(seed)
    xy = rng.uniform(-extent / 2 * 0.9, extent / 2 * 0.9, (2, n))
    z = rng.uniform(0.0, 0.3, n)
    means = np.concatenate([xy, z[None]], 0)
    scales = np.exp(rng.uniform(np.log(scale_range[0]), np.log(scale_range[1]), (2, n)))
    quats = scenegen._random_quats(rng, n, cap)
    op = rng.uniform(0.05, 0.95, n)
    rgb = rng.uniform(0, 1, (3, n))
    if oblique:
        cam = oblique_camera(rng, width=width, height=height, k=k,
                             off_nadir_deg=rng.uniform(5, 30), max_alt=1.0)
    else:
        cam = nadir_camera(width=width, height=height, k=k, max_alt=1.0)
    if delta:
        cam.dF_xy = np.concatenate([rng.normal(0, 0.3, (2, 3)), rng.normal(0, 0.5, (2, 1))],
                                   1).astype(np.float32)
    if color_noise:
        cam.color = (np.concatenate([np.eye(3), np.zeros((3, 1))], 1)
                     + rng.normal(0, color_noise, (3, 4))).astype(np.float32)
    cam.shadow_w, cam.shadow_h, cam.shadow_scale = width, height, 1.0
    return make(means, scales, quats, op, rgb, [cam])
