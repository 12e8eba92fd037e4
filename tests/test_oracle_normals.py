"""Pins of the FP64 depth-gradient normal oracle (Sec. 3.2 Eq. surface_normal), on the CPU.

Independent checks: a tilted plane seen through any affine camera gives the plane's own normal
(solved here from the camera and the plane, not through the oracle's point map), flat ground
gives +z, border and empty pixels give 0, and the hand-written adjoint matches central
differences."""
import numpy as np

import scenegen
from oracle import normals as NO

EPS = 1e-3


def _cam(seed, w=40, h=32, off=25.0):
    sc = scenegen.make_scene(n=16, extent_m=80.0, seed=seed,
                             views=[dict(width=w, height=h, off_nadir=off, delta=True)])
    return sc.cameras[0]


def _plane_depth(cam, a, b, c0):
    """Rendered depth (alpha = 1) of the plane h = a X + b Y + c0: for each pixel solve
    B'[:, :2] (X, Y) + B'[:, 2] h + b' = x together with the plane equation."""
    F = np.asarray(cam.F_xy, np.float32).astype(np.float64) + np.asarray(cam.dF_xy, np.float32).astype(np.float64)
    M = np.zeros((3, 3))
    M[:2, :] = F[:, :3]
    M[2, :] = [a, b, -1.0]
    H, W = cam.height, cam.width
    depth = np.zeros((H, W))
    maxalt = float(np.float32(cam.max_alt))
    for j in range(H):
        for i in range(W):
            rhs = np.array([i + 0.5 - F[0, 3], j + 0.5 - F[1, 3], -c0])
            X, Y, h = np.linalg.solve(M, rhs)
            depth[j, i] = maxalt - h
    return depth


def test_tilted_plane_gives_its_normal():
    for seed, (a, b) in [(1, (0.3, -0.2)), (2, (-0.5, 0.1)), (3, (0.0, 0.0))]:
        cam = _cam(seed)
        depth = _plane_depth(cam, a, b, 0.01)
        N, ok = NO.depth_normal(depth, np.ones_like(depth), cam, EPS)
        n_true = np.array([-a, -b, 1.0]) / np.linalg.norm([-a, -b, 1.0])
        assert ok[1:-1, 1:-1].all() and not ok[0].any() and not ok[:, -1].any()
        assert np.allclose(N[:, ok], n_true[:, None], atol=1e-12)
        assert np.all(N[:, ~ok] == 0.0)


def test_alpha_normalised_depth_and_empty_pixels():
    cam = _cam(4)
    depth = _plane_depth(cam, 0.2, 0.1, 0.0)
    alpha = np.full_like(depth, 0.6)
    alpha[10, 10] = 0.0  # no surface: it and its four neighbours get no normal
    N, ok = NO.depth_normal(depth * alpha, alpha, cam, EPS)
    n_true = np.array([-0.2, -0.1, 1.0]) / np.linalg.norm([-0.2, -0.1, 1.0])
    assert np.allclose(N[:, ok], n_true[:, None], atol=1e-12)
    for (j, i) in [(10, 10), (9, 10), (11, 10), (10, 9), (10, 11)]:
        assert not ok[j, i] and np.all(N[:, j, i] == 0.0)


def _smooth(rng, shape, lo, hi, n=5):
    yy, xx = np.mgrid[0:shape[0], 0:shape[1]] / max(shape)
    f = np.zeros(shape)
    for _ in range(n):
        p, q, r = rng.normal(size=3)
        f += np.sin(3 * p * xx + 3 * q * yy + r)
    f = (f - f.min()) / (f.max() - f.min() + 1e-12)
    return lo + (hi - lo) * f


def test_adjoint_matches_central_differences():
    cam = _cam(5, w=30, h=26)
    rng = np.random.default_rng(5)
    maxalt = float(np.float32(cam.max_alt))
    alpha = _smooth(rng, (cam.height, cam.width), 0.5, 1.0)
    depth = (maxalt - _smooth(rng, (cam.height, cam.width), 0.0, 0.01)) * alpha
    dF = np.asarray(cam.dF_xy, np.float64)
    w = rng.normal(size=(3, cam.height, cam.width))

    def loss(d_, a_, f_):
        N, _ = NO.depth_normal(d_, a_, cam, EPS, dF=f_)
        return float(np.sum(w * N))

    g = NO.depth_normal_backward(w, depth, alpha, cam, EPS, dF=dF)
    for key, h, base in (("depth", 1e-9, depth), ("alpha", 1e-7, alpha), ("dF", 1e-6, dF)):
        dirn = rng.normal(size=base.shape)
        args = dict(depth=depth, alpha=alpha, dF=dF)
        plus = dict(args); plus[key] = base + h * dirn
        minus = dict(args); minus[key] = base - h * dirn
        fd = (loss(plus["depth"], plus["alpha"], plus["dF"]) - loss(minus["depth"], minus["alpha"], minus["dF"])) / (2 * h)
        an = float(np.sum(g[key] * dirn))
        assert abs(fd - an) <= 1e-6 + 2e-3 * abs(an), (key, fd, an)
    # a translation of the camera moves no normal
    assert np.abs(g["dF"][:, 3]).max() < 1e-9 * max(1.0, np.abs(g["dF"]).max())
