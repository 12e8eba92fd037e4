"""Pins of the oracle's distortion plane (the point-sample distortion of the blending weights
along each ray, which the training loss of Supp. B adds), checked against closed forms on
hand-built stacks of flat splats and against invariances of the definition.  The adjoint of
the plane is checked against dual numbers and central differences with the rest of the
rasterizer adjoint in ``test_oracle_pins.py``."""
import math

import numpy as np
import pytest

import oracle
from tests import helpers as H


def _flat_stack(heights, scales, opacity, k=10.0, max_alt=2.0):
    """Flat (nadir-facing) splats, all centred on the image centre, given front to back."""
    cam = H.nadir_camera(16, 16, k=k, max_alt=max_alt)
    n = len(heights)
    sc = H.make([[0.0] * n, [0.0] * n, list(heights)], [list(scales), list(scales)],
                [[1] * n, [0] * n, [0] * n, [0] * n], list(opacity), np.full((3, n), 0.5), [cam])
    return cam, sc


def _weights_and_depths(sc, cam, i, j):
    """Closed form at pixel (i, j): the object-space Gaussian of each flat splat (it dominates
    the screen-space bound near the centre), alpha = o G, weights by front-to-back
    compositing in the given (height-descending) order, intersection depth max_alt - height."""
    k = float(cam.F_xy[0, 0])
    x, y = i + 0.5 - cam.width / 2, j + 0.5 - cam.height / 2
    w, z, T = [], [], 1.0
    for s in range(sc.opacity.shape[0]):
        su = float(sc.scales[0, s])
        g = math.exp(-0.5 * ((x / k / su) ** 2 + (y / k / su) ** 2))
        g_screen = math.exp(-(x * x + y * y) / (2 * oracle.Opts().sigma ** 2))
        assert g > g_screen
        a = float(sc.opacity[s]) * g
        assert oracle.Opts().alpha_min < a < oracle.Opts().alpha_max
        w.append(a * T)
        z.append(float(np.float32(cam.max_alt)) - float(sc.means[2, s]))
        T *= 1 - a
    return np.array(w), np.array(z)


def test_single_splat_has_no_distortion():
    sc = H.random_scene(5, n=1, width=24, height=20)
    out = oracle.render(oracle.SceneF64.of(sc), sc.cameras[0])
    assert out["alpha"].max() > 0.05
    assert np.all(out["distort"] == 0.0)


def test_two_stacked_splats_closed_form():
    """Two splats: 2 w_front w_back (z_back - z_front), with w_back = (1 - a_front) a_back."""
    cam, sc = _flat_stack([0.4, 0.1], [0.3, 0.25], [0.6, 0.7])
    out = oracle.render(oracle.SceneF64.of(sc), cam)
    for (i, j) in [(8, 8), (7, 8), (9, 6)]:
        w, z = _weights_and_depths(sc, cam, i, j)
        assert z[1] > z[0]
        expect = 2.0 * w[0] * w[1] * (z[1] - z[0])
        assert out["distort"][j, i] == pytest.approx(expect, rel=1e-12)


def test_sorted_stack_equals_the_unordered_pair_sum():
    """With the compositing order equal to the depth order, the plane is the point-sample
    distortion sum_{i,j} w_i w_j |z_i - z_j| over all ordered pairs."""
    cam, sc = _flat_stack([0.5, 0.4, 0.2, 0.05], [0.3, 0.2, 0.35, 0.25], [0.5, 0.4, 0.6, 0.8])
    out = oracle.render(oracle.SceneF64.of(sc), cam)
    for (i, j) in [(8, 8), (7, 7), (9, 8), (8, 10)]:
        w, z = _weights_and_depths(sc, cam, i, j)
        expect = float(np.sum(w[:, None] * w[None, :] * np.abs(z[:, None] - z[None, :])))
        assert out["distort"][j, i] == pytest.approx(expect, rel=1e-12)
        assert out["distort"][j, i] > 0


def test_coplanar_splats_have_no_distortion():
    """Splats that all lie in one horizontal plane meet every ray at one depth."""
    rng = np.random.default_rng(2)
    n = 12
    cam = H.nadir_camera(24, 24, k=12.0)
    xy = rng.uniform(-0.5, 0.5, (2, n))
    sc = H.make(np.concatenate([xy, np.full((1, n), 0.3)]), rng.uniform(0.1, 0.3, (2, n)),
                np.tile([[1.0], [0.0], [0.0], [0.0]], (1, n)), rng.uniform(0.3, 0.9, n),
                rng.uniform(0, 1, (3, n)), [cam])
    out = oracle.render(oracle.SceneF64.of(sc), cam)
    assert (out["ncontrib"] >= 2).sum() > 50
    assert np.abs(out["distort"]).max() <= 1e-12


def test_distortion_is_invariant_to_a_common_height_shift():
    """Moving every splat up by the same amount under a nadir camera leaves each ray's
    weights unchanged and shifts every intersection depth by the same amount: the distortion
    is unchanged while the depth plane moves by alpha times the shift."""
    sc = H.random_scene(7, n=30, width=32, height=28, oblique=False)
    cam = sc.cameras[0]
    assert float(cam.F_xy[0, 2]) == 0.0 and float(cam.F_xy[1, 2]) == 0.0
    s64 = oracle.SceneF64.of(sc)
    out = oracle.render(s64, cam)
    up = s64.means.copy()
    up[2] += 0.25
    out2 = oracle.render(oracle.SceneF64(up, s64.scales, s64.quats, s64.opacity, s64.rgb), cam)
    assert (out["ncontrib"] >= 2).sum() > 50
    np.testing.assert_allclose(out2["distort"], out["distort"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(out2["depth"], out["depth"] - 0.25 * out["alpha"], rtol=1e-9, atol=1e-12)
    assert np.abs(out["distort"]).max() > 1e-3
