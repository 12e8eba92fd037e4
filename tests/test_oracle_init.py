"""Pins of the geometry-aware initialisation oracle (Sec. 3.4), on CPU: closed forms of the area
weight and normal on flat, tilted and stepped DSMs, sampling statistics, the tangent-plane
jitter, the Gram-Schmidt basis, and the k-d tree kNN against brute force."""
import math

import numpy as np

import scenegen
from oracle import init as I
from oracle import optim as O


def _dsm(Z, gsd=0.01, rgb=None):
    Z = np.asarray(Z, np.float32)
    H, W = Z.shape
    rgb = np.full((3, H, W), 0.5, np.float32) if rgb is None else rgb
    return scenegen.DSM(height=Z, rgb=rgb, x0=float(np.float32(-0.5)), y0=float(np.float32(0.5)),
                        gsd=float(np.float32(gsd)), scale_m=1.0)


def test_vectorised_philox_equals_the_scalar_one():
    rng = np.random.default_rng(0)
    c = [rng.integers(0, 2 ** 63, 40, dtype=np.uint64) * 2 + rng.integers(0, 2, 40, dtype=np.uint64)
         for _ in range(4)]
    v = O.philox4x64_vec(*c, 2 ** 64 - 3, 77)
    for i in range(40):
        assert tuple(int(x[i]) for x in v) == O.philox4x64(tuple(int(x[i]) for x in c), (2 ** 64 - 3, 77))
    a = rng.integers(0, 2 ** 63, 200, dtype=np.uint64) * 2 + 1
    b = rng.integers(0, 2 ** 63, 200, dtype=np.uint64)
    h = O.mulhi64_vec(a, b)
    assert all(int(h[i]) == (int(a[i]) * int(b[i])) >> 64 for i in range(200))


def test_flat_dsm_weights_normals_and_basis():
    d = _dsm(np.full((6, 7), 0.2))
    w = I.weights(d)
    assert np.all(w == w[0, 0]) and abs(int(w[0, 0]) - 65536) <= 1
    n = I.normals(d)
    np.testing.assert_allclose(n, np.broadcast_to(np.array([0, 0, 1.0])[:, None, None], n.shape), atol=1e-15)
    tu, tv, nn = I.basis(d, np.arange(42))
    np.testing.assert_allclose(tu, np.tile([[1.0], [0], [0]], (1, 42)), atol=1e-15)
    np.testing.assert_allclose(tv, np.tile([[0.0], [1], [0]], (1, 42)), atol=1e-15)


def test_tilted_plane_closed_form():
    """Z = a x + b y: the area element sqrt(1 + a^2 + b^2) and the normal (-a, -b, 1) / norm."""
    a, b, g = 0.7, -0.3, 0.01
    H, W = 9, 11
    x = -0.5 + np.arange(W) * g
    y = 0.5 - np.arange(H) * g
    Z = a * x[None, :] + b * y[:, None]
    d = _dsm(Z, g)
    w = I.weights(d)
    expect = 65536 * math.sqrt(1 + a * a + b * b)
    assert np.all(np.abs(w[1:-1, 1:-1] - expect) <= 2 + 1e-5 * expect)
    n = I.normals(d)
    nz = np.array([-a, -b, 1.0]) / math.sqrt(1 + a * a + b * b)
    np.testing.assert_allclose(n[:, 1:-1, 1:-1].reshape(3, -1), np.tile(nz[:, None], (1, (H - 2) * (W - 2))),
                               atol=2e-5)  # the heights are float32
    tu, tv, nn = I.basis(d, np.arange(H * W))
    for t in (tu, tv, nn):
        np.testing.assert_allclose(np.linalg.norm(t, axis=0), 1.0, atol=1e-14)
    assert np.abs(np.sum(tu * tv, axis=0)).max() < 1e-14
    np.testing.assert_allclose(nn, I.normals(d).reshape(3, -1), atol=1e-12)


def test_facade_weight_closed_form():
    """A step of height h between columns 4 and 5: the two edge pixels see dz_x = h / 2 and weigh
    sqrt((h/2)^2 + g^2) / g flat pixels; the others weigh one."""
    g, h = 0.01, 0.3
    Z = np.zeros((5, 10), np.float32)
    Z[:, 5:] = h
    d = _dsm(Z, g)
    w = I.weights(d)
    zh = float(np.float32(np.float32(h) * np.float32(0.5)))
    expect = 65536 * math.sqrt(zh * zh + g * g) / g
    assert np.all(np.abs(w[:, 4:6] - expect) <= 1e-5 * expect + 2)
    assert np.all(np.abs(w[:, :4] - 65536) <= 1) and np.all(np.abs(w[:, 6:] - 65536) <= 1)


def test_draws_follow_the_weights_and_stay_in_the_tangent_plane():
    Z = np.zeros((6, 6), np.float32)
    Z[:, 3:] = 0.2  # a facade between columns 2 and 3
    d = _dsm(Z, 0.01)
    w = I.weights(d)
    n = 60000
    pix, u, v = I.draw_pixels(w, n, seed=4)
    freq = np.bincount(pix, minlength=36) / n
    p = w.reshape(-1) / w.sum()
    assert np.all(np.abs(freq - p) <= 5 * np.sqrt(p * (1 - p) / n))
    assert np.all(np.abs(u) < 0.5) and np.all(np.abs(v) < 0.5)
    assert abs(u.mean()) < 0.01 and abs(v.mean()) < 0.01
    out = I.init_splats(d, 400, seed=5)
    i, j = out["pixels"] % 6, out["pixels"] // 6
    g = d.gsd  # the float32 grid step, widened
    P = np.stack([-0.5 + i * g, 0.5 - j * g, Z.reshape(-1)[out["pixels"]].astype(np.float64)])
    nrm = I.normals(d).reshape(3, -1)[:, out["pixels"]]
    assert np.abs(np.sum((out["means"] - P) * nrm, axis=0)).max() < 1e-12
    # the rotation's third column is the DSM normal
    np.testing.assert_allclose(out["R"][:, 2, :], nrm, atol=1e-12)


def test_knn_equals_brute_force_and_a_lattice():
    rng = np.random.default_rng(6)
    p = rng.uniform(size=(3, 300))
    d = np.linalg.norm(p[:, :, None] - p[:, None, :], axis=0)
    np.fill_diagonal(d, np.inf)
    brute = np.sort(d, axis=1)[:, :3].mean(axis=1)
    np.testing.assert_allclose(I.knn_mean_distance(p, 3), brute, rtol=1e-12)
    # a square lattice of spacing s: every interior point has 4 neighbours at s
    s = 0.25
    gx, gy = np.meshgrid(np.arange(8) * s, np.arange(8) * s)
    lat = np.stack([gx.ravel(), gy.ravel(), np.zeros(64)])
    m = I.knn_mean_distance(lat, 3)
    interior = (gx.ravel() > 0) & (gx.ravel() < 7 * s) & (gy.ravel() > 0) & (gy.ravel() < 7 * s)
    np.testing.assert_allclose(m[interior], s, rtol=1e-12)


def test_quaternion_is_the_gram_schmidt_rotation():
    dsm = scenegen.make_dsm(size_px=64, extent_m=32.0, seed=3, n_buildings=3)
    out = I.init_splats(dsm, 500, seed=1)
    q = out["quats"] / np.linalg.norm(out["quats"], axis=0)
    R = O.rotation(q)
    np.testing.assert_allclose(R, out["R"], atol=1e-12)
    assert np.all(out["quats"][0] >= 0)
    assert np.all(out["scales"] > 0) and np.all(out["scales"][0] == out["scales"][1])
