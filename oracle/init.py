"""FP64 CPU oracle of the geometry-aware initialisation (Sec. 3.4): area-weighted sampling of
splat centres from a DSM, splat orientation from the DSM's local normal by Gram-Schmidt, and
splat scales from the mean distance to the k nearest sampled points.

TEST INFRASTRUCTURE ONLY: only the test-suite may import this module.  It shares no code with
the CUDA path; the CUDA path never imports it.

The DSM is a north-up grid: pixel (i, j) (column i, row j) is the point
P = (x0 + i g, y0 - j g, Z[j, i]).  Per pixel (Sec. 3.4):
  - tangents from finite differences of the neighbouring points, dx toward +x (the next
    column) and dy toward +y (the previous row): central differences inside, one-sided on the
    border, so that each spans one pixel: dx = (g, 0, dz_x), dy = (0, g, dz_y);
  - area weight a = |dx x dy| = g sqrt(dz_x^2 + dz_y^2 + g^2); normal n = (dx x dy) / a.
Readings where the paper is silent:
  - the weights are normalised as integers w = floor(sqrt(dz_x^2 + dz_y^2 + g^2) 2^16 / g) (a
    flat pixel weighs 2^16), computed in float32 in this order, so that the GPU and the oracle
    take every sampling decision identically; the probability of a pixel is w / sum(w);
  - sample j draws Philox4x64-10 with key (seed, 0) and counter (j, 0, 2, 0): the first word x
    picks the pixel as the last one whose exclusive prefix sum of weights is <= floor(x W / 2^64)
    (W the total), the next two give a jitter u, v = ((x >> 40) + 0.5) 2^-24 - 1/2 in the
    pixel's tangent plane: centre = P + u dx + v dy (samples of one pixel do not coincide);
  - the basis: t_u = dx / |dx|, t_v the Gram-Schmidt residual of dy against t_u, normalised,
    and the normal t_u x t_v (= n); the rotation [t_u t_v n] as a quaternion (w >= 0);
  - colour: the orthophoto at the pixel; opacity: a constant (0.1);
  - scales s_u = s_v = the mean Euclidean distance to the k (3) nearest other samples.
"""
from __future__ import annotations

import numpy as np

from . import optim as _philox_source  # the counter-based generator (Philox4x64-10) and uniforms

STREAM_INIT = 2


def _dz(Z):
    """dz_x (toward +x) and dz_y (toward +y, i.e. the previous row), float32, one pixel each."""
    Z = np.asarray(Z, np.float32)
    H, W = Z.shape
    dzx = np.zeros_like(Z)
    dzy = np.zeros_like(Z)
    half = np.float32(0.5)
    if W > 1:
        dzx[:, 1:-1] = (Z[:, 2:] - Z[:, :-2]) * half
        dzx[:, 0] = Z[:, 1] - Z[:, 0]
        dzx[:, -1] = Z[:, -1] - Z[:, -2]
    if H > 1:
        dzy[1:-1, :] = (Z[:-2, :] - Z[2:, :]) * half
        dzy[0, :] = Z[0, :] - Z[1, :]
        dzy[-1, :] = Z[-2, :] - Z[-1, :]
    return dzx, dzy


def weights(dsm) -> np.ndarray:
    """Integer area weights (H, W), int64, from float32 arithmetic in the stated order."""
    dzx, dzy = _dz(dsm.height)
    g = np.float32(dsm.gsd)
    q = (dzx * dzx + dzy * dzy) + g * g
    kscale = np.float32(65536.0 / float(g))
    w = np.floor(np.sqrt(q) * kscale)
    return np.minimum(w, np.float32(2 ** 31 - 1)).astype(np.int64)


def normals(dsm) -> np.ndarray:
    """Unit normals (3, H, W) in float64: (dx x dy) / |dx x dy|."""
    dzx, dzy = (a.astype(np.float64) for a in _dz(dsm.height))
    g = float(np.float32(dsm.gsd))
    c = np.stack([-g * dzx, -g * dzy, np.full_like(dzx, g * g)])
    return c / np.linalg.norm(c, axis=0)


def draw_pixels(w: np.ndarray, n: int, seed: int):
    """Pixel (flat index) and jitter (u, v) of every sample."""
    flat = w.reshape(-1).astype(np.int64)
    excl = np.concatenate([[0], np.cumsum(flat)[:-1]])  # exact in int64 (total < 2^63)
    total = int(flat.sum())
    j = np.arange(n, dtype=np.uint64)
    z = np.zeros(n, np.uint64)
    x0, x1, x2, _ = _philox_source.philox4x64_vec(j, z, np.full(n, STREAM_INIT, np.uint64), z, seed, 0)
    r = _philox_source.mulhi64_vec(x0, np.full(n, total, np.uint64)).astype(np.int64)
    pix = np.searchsorted(excl, r, side="right") - 1
    uni = lambda x: ((x >> np.uint64(40)).astype(np.float64) + 0.5) / float(1 << 24)
    return pix.astype(np.int64), uni(x1) - 0.5, uni(x2) - 0.5


def basis(dsm, pix: np.ndarray):
    """t_u, t_v, n (each (3, m)) at the given flat pixel indices, by Gram-Schmidt."""
    dzx, dzy = (a.astype(np.float64).reshape(-1)[pix] for a in _dz(dsm.height))
    g = float(np.float32(dsm.gsd))
    dx = np.stack([np.full_like(dzx, g), np.zeros_like(dzx), dzx])
    dy = np.stack([np.zeros_like(dzy), np.full_like(dzy, g), dzy])
    tu = dx / np.linalg.norm(dx, axis=0)
    r = dy - np.sum(dy * tu, axis=0) * tu
    tv = r / np.linalg.norm(r, axis=0)
    return tu, tv, np.cross(tu, tv, axis=0)


def knn_mean_distance(points: np.ndarray, k: int) -> np.ndarray:
    """Mean distance of each point (3, m) to its k nearest other points (scipy's k-d tree)."""
    from scipy.spatial import cKDTree
    p = np.asarray(points, np.float64).T
    d, _ = cKDTree(p).query(p, k=k + 1)
    return d[:, 1:].mean(axis=1)


def init_splats(dsm, n: int, seed: int = 0, k: int = 3, opacity: float = 0.1, index=None):
    """The initial splats: dict of means (3, n), scales (2, n), quats (4, n) (w, x, y, z),
    opacity (n,), rgb (3, n), and the drawn pixels.  `index` restricts the per-sample
    attributes to those samples (the kNN still runs over all n)."""
    from scipy.spatial.transform import Rotation
    w = weights(dsm)
    H, W = w.shape
    pix, u, v = draw_pixels(w, n, seed)
    i, j = pix % W, pix // W
    dzx, dzy = (a.astype(np.float64).reshape(-1)[pix] for a in _dz(dsm.height))
    g = float(np.float32(dsm.gsd))
    Z = np.asarray(dsm.height, np.float64).reshape(-1)[pix]
    means = np.stack([float(np.float32(dsm.x0)) + (i + u) * g,
                      float(np.float32(dsm.y0)) - j * g + v * g,
                      Z + u * dzx + v * dzy])
    s = knn_mean_distance(means, k)
    sel = np.arange(n) if index is None else np.asarray(index)
    tu, tv, nn = basis(dsm, pix[sel])
    R = np.stack([tu, tv, nn], axis=1)  # (3, 3, m): columns t_u, t_v, n
    q = Rotation.from_matrix(np.moveaxis(R, 2, 0)).as_quat()  # (m, 4) x, y, z, w
    q = np.stack([q[:, 3], q[:, 0], q[:, 1], q[:, 2]])
    q = q * np.where(q[0] < 0, -1.0, 1.0)
    rgb = np.asarray(dsm.rgb, np.float64).reshape(3, -1)[:, pix[sel]]
    return dict(means=means[:, sel], scales=np.stack([s[sel], s[sel]]), quats=q,
                opacity=np.full(len(sel), opacity), rgb=rgb, pixels=pix[sel], R=R)
