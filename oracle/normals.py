"""FP64 CPU oracle of the depth-gradient surface normal (Sec. 3.2 Eq. surface_normal).

TEST INFRASTRUCTURE ONLY: like the rest of ``oracle/``, only the test-suite may import it.  It
shares no code with the CUDA path.  Plain numpy in float64 over the pixels of one view, with the
adjoint written out by hand.

N = (grad_x p_s x grad_y p_s) / |grad_x p_s x grad_y p_s|, p_s the 3-D point map back-projected
from the depth map, in world coordinates (an affine camera does not keep screen-space angles).
Readings where the paper is silent:
  - the depth of a pixel is its alpha-normalised rendered depth z = D / alpha, its height
    h = max_alt - z (depth row B_z = [0, 0, -1], b_z = max_alt);
  - p_s(x) = (X, Y, h) with B'[:, 0:2] (X, Y) = x - b' - B'[:, 2] h (the main camera inverted at
    that height; B' = F'[:, 0:3], b' = F'[:, 3]);
  - grad_x p_s = p_s(i + 1, j) - p_s(i - 1, j), grad_y p_s = p_s(i, j + 1) - p_s(i, j - 1)
    (central differences; the scale cancels in the normalisation);
  - N is multiplied by sign(det B'[:, 0:2]), so that flat ground gets (0, 0, 1) whatever the
    orientation of the image axes (up, toward the sensor, as the rendered normals);
  - a pixel on the image border, or with a neighbour or itself without a surface
    (alpha < eps), has N = 0.
"""
from __future__ import annotations

import numpy as np


def _camera(cam, dF):
    F = np.asarray(cam.F_xy, np.float32).astype(np.float64)
    d = np.asarray(cam.dF_xy, np.float32).astype(np.float64) if dF is None else np.asarray(dF, np.float64)
    Fp = F + d
    return Fp[:, :3], Fp[:, 3]


def point_map(depth, alpha, cam, eps, dF=None):
    """p_s (3, H, W) and the surface mask (alpha >= eps)."""
    B, b = _camera(cam, dF)
    A = B[:, :2]
    H, W = depth.shape
    y, x = np.mgrid[0:H, 0:W].astype(np.float64) + 0.5
    surf = alpha >= eps
    z = np.where(surf, depth / np.where(surf, alpha, 1.0), 0.0)
    h = float(np.float32(cam.max_alt)) - z
    rhs = np.stack([x - b[0] - B[0, 2] * h, y - b[1] - B[1, 2] * h])
    XY = np.linalg.solve(A, rhs.reshape(2, -1)).reshape(2, H, W)
    return np.stack([XY[0], XY[1], h]), surf


def depth_normal(depth, alpha, cam, eps, dF=None):
    """N (3, H, W) of one view from its rendered depth and alpha."""
    P, surf = point_map(depth, alpha, cam, eps, dF)
    B, _ = _camera(cam, dF)
    sgn = np.sign(np.linalg.det(B[:, :2]))
    H, W = depth.shape
    N = np.zeros((3, H, W))
    ok = np.zeros((H, W), bool)
    ok[1:-1, 1:-1] = surf[1:-1, 1:-1] & surf[1:-1, 2:] & surf[1:-1, :-2] & surf[2:, 1:-1] & surf[:-2, 1:-1]
    gx = P[:, 1:-1, 2:] - P[:, 1:-1, :-2]
    gy = P[:, 2:, 1:-1] - P[:, :-2, 1:-1]
    c = np.cross(gx, gy, axis=0)
    n = np.linalg.norm(c, axis=0)
    inner = np.where(ok[1:-1, 1:-1], sgn * c / np.where(n > 0, n, 1.0), 0.0)
    N[:, 1:-1, 1:-1] = inner
    return N, ok


def depth_normal_backward(dN, depth, alpha, cam, eps, dF=None):
    """Adjoint of depth_normal for the upstream gradient dN (3, H, W): d_depth, d_alpha and
    d_dF (2, 4)."""
    B, b = _camera(cam, dF)
    A = B[:, :2]
    Ainv = np.linalg.inv(A)
    sgn = np.sign(np.linalg.det(A))
    P, surf = point_map(depth, alpha, cam, eps, dF)
    H, W = depth.shape
    ok = np.zeros((H, W), bool)
    ok[1:-1, 1:-1] = surf[1:-1, 1:-1] & surf[1:-1, 2:] & surf[1:-1, :-2] & surf[2:, 1:-1] & surf[:-2, 1:-1]
    gx = P[:, 1:-1, 2:] - P[:, 1:-1, :-2]
    gy = P[:, 2:, 1:-1] - P[:, :-2, 1:-1]
    c = np.cross(gx, gy, axis=0)
    n = np.linalg.norm(c, axis=0)
    m = ok[1:-1, 1:-1]
    nn = np.where(m, n, 1.0)
    Nin = c / nn
    d = np.where(m, dN[:, 1:-1, 1:-1], 0.0)
    # N = sgn c / |c|: dc = sgn (dN - N (N . dN)) / |c|
    dc = sgn * (d - Nin * np.sum(Nin * d, axis=0)) / nn
    # c = gx x gy: d gx = gy x dc, d gy = dc x gx
    dgx = np.cross(gy, dc, axis=0)
    dgy = np.cross(dc, gx, axis=0)
    dP = np.zeros_like(P)
    dP[:, 1:-1, 2:] += dgx
    dP[:, 1:-1, :-2] -= dgx
    dP[:, 2:, 1:-1] += dgy
    dP[:, :-2, 1:-1] -= dgy
    # P = (X, Y, h), (X, Y) = A^-1 (x - b' - B'[:, 2] h)
    dXY = dP[:2]
    # d h = dP_z + (A^-1 B'[:, 2] ... ) : dX/dh = -A^-1 B'[:, 2]
    g = -Ainv @ B[:, 2]
    dh = dP[2] + g[0] * dXY[0] + g[1] * dXY[1]
    # d A^-1 and d B'[:, 2], d b' (b' does not move the normal, its derivative sums to zero
    # only in exact arithmetic: it is kept)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64) + 0.5
    h = P[2]
    rhs = np.stack([x - b[0] - B[0, 2] * h, y - b[1] - B[1, 2] * h])
    dAinv = np.einsum("ihw,jhw->ij", dXY, rhs)
    drhs = np.einsum("ij,ihw->jhw", Ainv, dXY)
    d_dF = np.zeros((2, 4))
    d_dF[0, 2] = np.sum(-drhs[0] * h)
    d_dF[1, 2] = np.sum(-drhs[1] * h)
    d_dF[0, 3] = np.sum(-drhs[0])
    d_dF[1, 3] = np.sum(-drhs[1])
    # A^-1: dA = -A^-T dAinv A^-T
    dA = -Ainv.T @ dAinv @ Ainv.T
    d_dF[:, :2] += dA
    # h = max_alt - z, z = D / alpha
    dz = -dh
    a_safe = np.where(surf, alpha, 1.0)
    d_depth = np.where(surf, dz / a_safe, 0.0)
    d_alpha = np.where(surf, -dz * depth / (a_safe * a_safe), 0.0)
    return dict(depth=d_depth, alpha=d_alpha, dF=d_dF)
