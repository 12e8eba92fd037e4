"""The tolerances of tests/tolerances.py that depart from the default rule are forced by FP32: the
FP64 oracle itself, run on inputs that carry errors of the size FP32 arithmetic commits, breaks the
default bound and stays within the departed one.  CPU only (oracle and numpy)."""
import numpy as np

import oracle
import scenegen
from oracle import normals as NO
from oracle import shade as S
from tests.tolerances import CHAIN_GRAD_FLOOR, FP32_PLANE_ERROR, NORMAL_FWD_TOL, NORMAL_GRAD_FLOOR

EPS = 1e-3
KEYS = ("means", "scales", "quats", "opacity", "rgb")


def outside(g, ref, floor, rtol=1e-3):
    """Number of elements outside the per-element bound 1e-3 (|ref| + floor max|ref|)."""
    g, ref = np.ravel(g), np.ravel(ref)
    scale = np.abs(ref).max()
    return int((np.abs(g - ref) > rtol * (np.abs(ref) + floor * scale)).sum())


def test_depth_normal_bounds():
    """The depth-normal kernels receive FP32 depth and alpha planes, exactly as the oracle does,
    and their first operation, z = D / alpha, is rounded to FP32.  One rounding of z (a relative
    error below 2^-24) moves the oracle's normal beyond the default 1e-5 and its depth and alpha
    gradients beyond the default per-element floor; the departed bounds hold."""
    scene = scenegen.make_scene(n=64, extent_m=400.0, seed=33, views=[
        dict(width=400, height=360, off_nadir=18.0, delta=True),
        dict(width=300, height=420, off_nadir=27.0, delta=False)])
    rng = np.random.default_rng(34)
    fwd_max, n_default, n_departed = 0.0, 0, 0
    for cam in scene.cameras:
        # the planes of the GPU test: a smooth height field with holes, alpha in [0.05, 1]
        y, x = np.mgrid[0:cam.height, 0:cam.width].astype(np.float64)
        z = 1.0 + 0.2 * np.sin(x / 37.0) * np.cos(y / 53.0) + 0.05 * np.sin((x + 2 * y) / 11.0)
        a = rng.uniform(0.05, 1.0, z.shape)
        a[rng.uniform(size=z.shape) < 0.02] = 0.0
        a = a.astype(np.float32).astype(np.float64)
        d = (a * z).astype(np.float32).astype(np.float64)
        dN = rng.normal(size=(3, cam.height, cam.width)).astype(np.float32).astype(np.float64)
        N, _ = NO.depth_normal(d, a, cam, EPS)
        g = NO.depth_normal_backward(dN, d, a, cam, EPS)
        for _ in range(2):
            dz = d * (1.0 + rng.uniform(-1.0, 1.0, d.shape) * 2.0 ** -24)  # z = D / alpha rounded
            N2, _ = NO.depth_normal(dz, a, cam, EPS)
            g2 = NO.depth_normal_backward(dN, dz, a, cam, EPS)
            fwd_max = max(fwd_max, float(np.abs(N2 - N).max()))
            for k in ("depth", "alpha"):
                n_default += outside(g2[k], g[k], 1e-3)
                n_departed += outside(g2[k], g[k], NORMAL_GRAD_FLOOR)
    assert 1e-5 < fwd_max <= NORMAL_FWD_TOL, fwd_max
    assert n_default > 0 and n_departed == 0, (n_default, n_departed)


def _chain_counts(chain, planes, seeds):
    """Elements outside the default and the departed floor, over seeds, when the chain runs on
    planes carrying absolute errors of FP32_PLANE_ERROR."""
    ref = chain(*planes)
    n_default = n_departed = 0
    for s in seeds:
        rng = np.random.default_rng(s)
        r2 = chain(*[p + rng.uniform(-FP32_PLANE_ERROR, FP32_PLANE_ERROR, p.shape) for p in planes])
        n_default += sum(outside(r2[k], ref[k], 1e-3) for k in KEYS)
        n_departed += sum(outside(r2[k], ref[k], CHAIN_GRAD_FLOOR) for k in KEYS)
    return n_default, n_departed


def test_normal_consistency_chain_bound():
    """The chain render -> depth_normal -> loss of the GPU test, run in FP64 on the oracle's planes
    and on the same planes with FP32-sized errors: the splat gradients leave the default
    per-element floor, not the departed one."""
    scene = scenegen.make_scene(n=2500, extent_m=50.0, seed=32, views=[
        dict(width=72, height=60, off_nadir=16.0, delta=True, color_noise=0.02)])
    cam = scene.cameras[0]
    s64 = oracle.SceneF64.of(scene)
    om = oracle.render(s64, cam, color=cam.color)
    w = np.random.default_rng(8).normal(size=(cam.height, cam.width))

    def chain(depth, alpha, normal):
        N, _ = NO.depth_normal(depth, alpha, cam, EPS)
        gN = NO.depth_normal_backward(-w[None] * normal, depth, alpha, cam, EPS)
        up = dict(alpha=w + gN["alpha"], depth=gN["depth"], normal=-w[None] * N)
        return oracle.backward(s64, cam, up, color=cam.color)

    n_default, n_departed = _chain_counts(chain, (om["depth"], om["alpha"], om["normal"]), range(200, 204))
    assert n_default > 0 and n_departed == 0, (n_default, n_departed)


def test_shade_chain_bound():
    """The chain render -> shade -> loss of the GPU test (sun visibility with k = 60), run in FP64
    on the oracle's main and sun planes and on the same planes with FP32-sized errors."""
    scene = scenegen.make_scene(n=3000, extent_m=60.0, seed=24, views=[
        dict(width=80, height=64, off_nadir=18.0, delta=True, color_noise=0.02)])
    cam = scene.cameras[0]
    s64 = oracle.SceneF64.of(scene)
    om = oracle.render(s64, cam, sun=False, color=cam.color)
    osn = oracle.render(s64, cam, sun=True)
    wI = np.random.default_rng(9).normal(size=(3, cam.height, cam.width))
    La = np.array([0.3, 0.35, 0.4])

    def chain(rgb, depth, alpha, sun_depth, sun_alpha):
        gs = S.shade_backward(wI, rgb, depth, alpha, sun_depth, sun_alpha, cam, La, 60.0, 0.0, EPS)
        gm = oracle.backward(s64, cam, dict(rgb=gs["rgb"], depth=gs["depth"], alpha=gs["alpha"]), color=cam.color)
        gsun = oracle.backward(s64, cam, dict(depth=gs["sun_depth"], alpha=gs["sun_alpha"]), sun=True)
        return {k: gm[k] + gsun[k] for k in KEYS}

    planes = (om["rgb"], om["depth"], om["alpha"], osn["depth"], osn["alpha"])
    n_default, n_departed = _chain_counts(chain, planes, range(100, 108))
    assert n_default > 0 and n_departed == 0, (n_default, n_departed)
