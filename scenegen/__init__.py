"""Seeded synthetic satellite scenes: splats, affine cameras, sun angles.

This module only draws random inputs.  It holds none of the rasterizer's
arithmetic: no projection, no camera assembly, no compositing.  Both the CUDA
path and the FP64 oracle consume what it returns.

World frame.  The paper works in normalised UTM coordinates (Sec. 3.1, the
affine camera paragraph; Supp. B).  Scenes are drawn in metres with the
distributions stated below and then mapped to the world frame by one isotropic
scale: ``world = metres / scale_m`` with ``scale_m`` = half the scene extent, so
x, y lie in [-1, 1] and heights keep their proportion to the ground extent.

Recipe (sizes per workload are in ``WORKLOADS``):
  * centres x, y ~ U[-E/2, E/2] m; z = h(x, y) + N(0, 0.5) m where h is a sum
    of 16 Gaussian bumps (random centres, widths 20-200 m) plus a low-frequency
    sinusoid, rescaled to [0, 20] m;
  * scales s_u, s_v independent, log-uniform on [0.5, 3] m;
  * rotations: normal uniform on the spherical cap within 30 deg of +z,
    in-plane angle uniform; stored as an unnormalised quaternion (w, x, y, z)
    with w >= 0 and a random norm in [0.5, 2];
  * opacity = sigmoid(N(0, 1)); rgb ~ U[0, 1]^3;
  * cameras: orthographic view along a direction at off-nadir angle theta_v,
    azimuth U[0, 2 pi); image axes perpendicular to it, image y pointing as
    close to south as possible; 0.5 m ground sampling distance; the view's
    target point maps to the image centre;
  * camera deltas (when enabled): N(0, 1e-3) px/m on the 2x3 block,
    N(0, 0.5) px on the offset;
  * colour correction: identity, optionally + N(0, 0.02) on all 12 entries;
  * sun: elevation U[40, 70] deg, azimuth U[0, 360) deg; shadow map at half
    the view's resolution (scale 0.5);
  * max_altitude = 30 m.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

GSD_M = 0.5          # metres per pixel
MAX_ALT_M = 30.0     # b_z of the depth row, metres


@dataclasses.dataclass
class Camera:
    """One affine view.  All float fields are float32 values as the kernels see them."""
    F_xy: np.ndarray        # (2, 4) world -> pixel, pixel (i, j) centre at (i + .5, j + .5)
    dF_xy: np.ndarray       # (2, 4) learnable delta
    max_alt: float          # b_z (world units)
    width: int
    height: int
    color: np.ndarray       # (3, 4) [C | c]
    sun_phi: float          # sun azimuth, radians
    sun_theta: float        # sun elevation, radians
    shadow_w: int
    shadow_h: int
    shadow_scale: float


@dataclasses.dataclass
class Scene:
    means: np.ndarray       # (3, N) float32, world units
    scales: np.ndarray      # (2, N) float32, world units, > 0
    quats: np.ndarray       # (4, N) float32, (w, x, y, z), unnormalised
    opacity: np.ndarray     # (N,) float32 in (0, 1)
    rgb: np.ndarray         # (3, N) float32
    cameras: List[Camera]
    scale_m: float          # metres per world unit
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.means.shape[1])


def _f32(x):
    return np.asarray(x, dtype=np.float32)


def _height_field(rng: np.random.Generator, extent: float):
    """Smooth seeded height function h(x, y) in metres, range [0, 20]."""
    nb = 16
    cx = rng.uniform(-extent / 2, extent / 2, nb)
    cy = rng.uniform(-extent / 2, extent / 2, nb)
    wd = rng.uniform(20.0, 200.0, nb)
    amp = rng.uniform(0.3, 1.0, nb)
    kx, ky = rng.uniform(0.5, 1.5, 2) * (2 * math.pi / extent)
    ph = rng.uniform(0, 2 * math.pi, 2)

    def raw(x, y):
        h = np.zeros_like(x, dtype=np.float64)
        for i in range(nb):
            h += amp[i] * np.exp(-((x - cx[i]) ** 2 + (y - cy[i]) ** 2) / (2 * wd[i] ** 2))
        h += 0.3 * np.sin(kx * x + ph[0]) * np.cos(ky * y + ph[1])
        return h

    gx, gy = np.meshgrid(np.linspace(-extent / 2, extent / 2, 65),
                         np.linspace(-extent / 2, extent / 2, 65))
    g = raw(gx, gy)
    lo, hi = float(g.min()), float(g.max())
    span = max(hi - lo, 1e-9)
    return lambda x, y: (raw(x, y) - lo) / span * 20.0


def _quat_mul(a, b):
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw])


def _random_quats(rng: np.random.Generator, n: int, cap_deg: float = 30.0):
    """Quaternions whose rotated +z lies in a cap around +z, random in-plane angle."""
    cos_t = rng.uniform(math.cos(math.radians(cap_deg)), 1.0, n)
    tilt = np.arccos(cos_t)
    az = rng.uniform(0, 2 * math.pi, n)
    psi = rng.uniform(0, 2 * math.pi, n)
    # in-plane spin about z, then tilt about the horizontal axis (-sin az, cos az, 0)
    q_spin = np.stack([np.cos(psi / 2), np.zeros(n), np.zeros(n), np.sin(psi / 2)])
    q_tilt = np.stack([np.cos(tilt / 2), -np.sin(az) * np.sin(tilt / 2),
                       np.cos(az) * np.sin(tilt / 2), np.zeros(n)])
    q = _quat_mul(q_tilt, q_spin)
    q *= np.where(q[0] < 0, -1.0, 1.0)
    q *= rng.uniform(0.5, 2.0, n)
    return q


def make_splats(rng: np.random.Generator, n: int, extent_m: float, scale_m: float):
    h = _height_field(rng, extent_m)
    x = rng.uniform(-extent_m / 2, extent_m / 2, n)
    y = rng.uniform(-extent_m / 2, extent_m / 2, n)
    z = h(x, y) + rng.normal(0.0, 0.5, n)
    su = np.exp(rng.uniform(math.log(0.5), math.log(3.0), n))
    sv = np.exp(rng.uniform(math.log(0.5), math.log(3.0), n))
    q = _random_quats(rng, n)
    op = 1.0 / (1.0 + np.exp(-rng.normal(0.0, 1.0, n)))
    rgb = rng.uniform(0.0, 1.0, (3, n))
    means = _f32(np.stack([x, y, z]) / scale_m)
    scales = _f32(np.stack([su, sv]) / scale_m)
    return means, scales, _f32(q), _f32(op), _f32(rgb)


def make_camera(rng: np.random.Generator, *, width: int, height: int, scale_m: float,
                off_nadir_deg: float, target_m=(0.0, 0.0, 0.0), delta: bool = False,
                color_noise: float = 0.0, shadow_scale: float = 0.5) -> Camera:
    """Orthographic affine view with world->pixel matrix F_xy (2 x 4)."""
    th = math.radians(off_nadir_deg)
    az = rng.uniform(0, 2 * math.pi)
    d = np.array([math.sin(th) * math.cos(az), math.sin(th) * math.sin(az), math.cos(th)])
    south = np.array([0.0, -1.0, 0.0])
    e2 = south - south.dot(d) * d
    e2 /= np.linalg.norm(e2)
    e1 = np.cross(d, e2)
    k = scale_m / GSD_M                      # pixels per world unit
    B = k * np.stack([e1, e2])               # (2, 3)
    T = np.asarray(target_m, dtype=np.float64) / scale_m
    b = np.array([width / 2.0, height / 2.0]) - B @ T
    F = np.concatenate([B, b[:, None]], axis=1)
    dF = np.zeros((2, 4))
    if delta:
        dF[:, :3] = rng.normal(0.0, 1e-3, (2, 3)) * scale_m
        dF[:, 3] = rng.normal(0.0, 0.5, 2)
    color = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    if color_noise > 0:
        color = color + rng.normal(0.0, color_noise, (3, 4))
    sun_el = math.radians(rng.uniform(40.0, 70.0))
    sun_az = rng.uniform(0.0, 2 * math.pi)
    sw = max(1, int(round(width * shadow_scale)))
    sh = max(1, int(round(height * shadow_scale)))
    return Camera(F_xy=_f32(F), dF_xy=_f32(dF), max_alt=float(np.float32(MAX_ALT_M / scale_m)),
                  width=int(width), height=int(height), color=_f32(color),
                  sun_phi=float(np.float32(sun_az)), sun_theta=float(np.float32(sun_el)),
                  shadow_w=sw, shadow_h=sh, shadow_scale=float(np.float32(shadow_scale)))


def make_scene(*, n: int, extent_m: float, views: List[dict], seed: int = 0, name: str = "") -> Scene:
    """``views``: dicts with width, height, off_nadir (deg or (lo, hi)), delta, color_noise,
    target ('centre' or 'random')."""
    scale_m = extent_m / 2.0
    rng = np.random.default_rng(seed)
    means, scales, quats, op, rgb = make_splats(rng, n, extent_m, scale_m)
    cams = []
    for i, v in enumerate(views):
        vr = np.random.default_rng(seed + 1000 + i)
        on = v.get("off_nadir", 15.0)
        if isinstance(on, (tuple, list)):
            on = vr.uniform(on[0], on[1])
        W, H = int(v["width"]), int(v["height"])
        if v.get("target", "centre") == "random":
            # keep the view's ground footprint inside the extent where possible
            half_x = max(0.0, extent_m / 2 - W * GSD_M / 2)
            half_y = max(0.0, extent_m / 2 - H * GSD_M / 2)
            tgt = (vr.uniform(-half_x, half_x), vr.uniform(-half_y, half_y), 10.0)
        else:
            tgt = (0.0, 0.0, 10.0)
        cams.append(make_camera(vr, width=W, height=H, scale_m=scale_m, off_nadir_deg=on,
                                target_m=tgt, delta=bool(v.get("delta", False)),
                                color_noise=float(v.get("color_noise", 0.0)),
                                shadow_scale=float(v.get("shadow_scale", 0.5))))
    return Scene(means, scales, quats, op, rgb, cams, scale_m, name)


# --------------------------------------------------------------------------------------------
# Named workloads (sizes of the paper-scale synthetic benchmarks)
# --------------------------------------------------------------------------------------------

def _uneven_sizes(seed: int, nviews: int):
    r = np.random.default_rng(seed + 77)
    choices = np.arange(1024, 2048 + 1, 64)
    return [(int(r.choice(choices)), int(r.choice(choices))) for _ in range(nviews)]


def workload(name: str, seed: int = 0, n: Optional[int] = None) -> Scene:
    """Scenes for the five standard workloads.

    small   : 4,096 splats, 100 m extent, one 128 x 128 view, 15 deg off-nadir.
    single  : 500k splats, 1 km extent, one 2048^2 view (5-30 deg), 1024^2 shadow map,
              colour correction near identity.
    batched : 1M splats, 1 km extent, 16 views of uneven size 1024^2-2048^2 with camera
              deltas; shadow maps at half resolution.
    bf16    : as 'single' (storage precision is chosen by the caller).
    full    : 4M splats, 2 km extent, 32 views at 2048^2 with 1024^2 shadow maps,
              deltas and colour correction.
    """
    if name == "small":
        return make_scene(n=n or 4096, extent_m=100.0, seed=seed, name=name,
                          views=[dict(width=128, height=128, off_nadir=15.0)])
    if name in ("single", "bf16"):
        return make_scene(n=n or 500_000, extent_m=1000.0, seed=seed, name=name,
                          views=[dict(width=2048, height=2048, off_nadir=(5.0, 30.0),
                                      color_noise=0.02)])
    if name == "batched":
        sizes = _uneven_sizes(seed, 16)
        return make_scene(n=n or 1_000_000, extent_m=1000.0, seed=seed, name=name,
                          views=[dict(width=w, height=h, off_nadir=(5.0, 30.0), delta=True,
                                      target="random") for (w, h) in sizes])
    if name == "full":
        return make_scene(n=n or 4_000_000, extent_m=2000.0, seed=seed, name=name,
                          views=[dict(width=2048, height=2048, off_nadir=(5.0, 30.0), delta=True,
                                      color_noise=0.02, target="random") for _ in range(32)])
    raise ValueError(f"unknown workload {name!r}")


@dataclasses.dataclass
class DSM:
    """A digital surface model on a north-up grid (world units): pixel (i, j) (column i, row j)
    is the point (x0 + i gsd, y0 - j gsd, height[j, i]); rgb is its orthophoto colour."""
    height: np.ndarray  # (H, W) float32
    rgb: np.ndarray     # (3, H, W) float32
    x0: float
    y0: float
    gsd: float
    scale_m: float


def make_dsm(*, size_px: int, extent_m: float, seed: int = 0, n_buildings: Optional[int] = None) -> DSM:
    """A seeded synthetic DSM of a built-up area, in the world frame of ``make_scene``
    (world = metres / (extent / 2)).

    Recipe: the smooth terrain of ``make_splats`` (0-20 m); axis-aligned rectangular buildings
    (footprints U[10, 60] m per side, heights U[5, 30] m above the terrain at their centre,
    flat roofs), about one per 50 x 50 m; orthophoto: terrain colour a smooth function of
    position plus N(0, 0.03) noise, one uniform colour per roof."""
    rng = np.random.default_rng(seed)
    scale_m = extent_m / 2.0
    h = _height_field(rng, extent_m)
    gsd_m = extent_m / size_px
    c = (np.arange(size_px) + 0.5) * gsd_m - extent_m / 2
    X, Y = np.meshgrid(c, -c)  # row j goes south
    Z = h(X, Y)
    rgb = np.stack([0.35 + 0.15 * np.sin(X / 37.0), 0.40 + 0.10 * np.cos(Y / 53.0),
                    0.30 + 0.10 * np.sin((X + Y) / 71.0)])
    rgb = rgb + rng.normal(0.0, 0.03, rgb.shape)
    nb = n_buildings if n_buildings is not None else max(1, int((extent_m / 50.0) ** 2))
    for _ in range(nb):
        cx, cy = rng.uniform(-extent_m / 2, extent_m / 2, 2)
        wx, wy = rng.uniform(10.0, 60.0, 2)
        top = float(h(np.array([cx]), np.array([cy]))[0]) + rng.uniform(5.0, 30.0)
        col = rng.uniform(0.2, 0.9, 3)
        # the pixels whose centres lie in the footprint (columns by x, rows by -y)
        i0 = int(np.searchsorted(c, cx - wx / 2, side="left"))
        i1 = int(np.searchsorted(c, cx + wx / 2, side="right"))
        j0 = int(np.searchsorted(c, -(cy + wy / 2), side="left"))
        j1 = int(np.searchsorted(c, -(cy - wy / 2), side="right"))
        if i0 >= i1 or j0 >= j1:
            continue
        Z[j0:j1, i0:i1] = np.maximum(Z[j0:j1, i0:i1], top)
        rgb[:, j0:j1, i0:i1] = col[:, None, None]
    return DSM(height=_f32(Z / scale_m), rgb=_f32(np.clip(rgb, 0.0, 1.0)),
               x0=float(np.float32(c[0] / scale_m)), y0=float(np.float32(-c[0] / scale_m)),
               gsd=float(np.float32(gsd_m / scale_m)), scale_m=scale_m)


def to_bf16_exact(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest-even) and return them widened back to
    float32, i.e. exactly the values a BF16 store holds."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(x.shape)


def upstream_grads(rng: np.random.Generator, height: int, width: int, sun: bool = False):
    """Seeded upstream gradients for the rendered planes of one view:
    (rgb (3,H,W), depth (H,W), normal (3,H,W), alpha (H,W)); sun views: depth, alpha."""
    g = lambda *s: rng.normal(0.0, 1.0, s).astype(np.float32)
    if sun:
        return None, g(height, width), None, g(height, width)
    return g(3, height, width), g(height, width), g(3, height, width), g(height, width)
