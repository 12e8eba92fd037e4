"""FP64 CPU oracle of the affine 2DGS rasterizer: Python loader (ctypes).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (the CUDA library and its binding) never imports it, and it never
imports the product path: inputs come from ``scenegen`` and every value is
converted exactly to float64 here.

The C++ source (``satsplat_oracle.cpp``) is the plain per-pixel definition of
Sec. 3.2 (Eq. affine2dgs_Qq, Eq. depth_affine_camera, Eq. rasterization), the
camera delta and sun camera of Sec. 3.3 / Supp. A (Eq. sun_camera_Bxy) and the
colour correction of Sec. 3.1 (Eq. image_formation), with a hand-written
reverse-mode adjoint and a dual-number forward mode that checks it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "satsplat_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# camera record layout (float64), matches the C++ enum
C_F, C_DF, C_MAXALT, C_W, C_H, C_COLOR, C_PHI, C_THETA, C_SW, C_SH, C_SSCALE, C_NUM = (
    0, 8, 16, 17, 18, 19, 31, 32, 33, 34, 35, 36)


def build(force: bool = False) -> str:
    """Compile the oracle with the host compiler (plain C++17 + OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            I64, I32 = ctypes.c_int64, ctypes.c_int
            L.ora_camera.argtypes = [P, I32, P, P, P, P]
            L.ora_project.argtypes = [I64, P, P, P, P, P, P, I32, P, P]
            L.ora_order.argtypes = [I64, P, P]
            L.ora_render.argtypes = [I64, P, P, P, P, P, P, I32, P, P, I32, I32, I32, I32, I32] + [P] * 10
            L.ora_render_dual.argtypes = ([I64, P, P, P, P, P, P, I32, P, P, I32, I32, I32, I32, I32]
                                          + [P] * 7 + [P] * 5)
            L.ora_backward.argtypes = ([I64, P, P, P, P, P, P, I32, P, P, I32, I32, I32, I32, I32]
                                       + [P] * 5 + [P] * 7)
            L.ora_num_threads.restype = I32
            L.ora_set_threads.argtypes = [I32]
            _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


@dataclass
class Opts:
    """Rasterizer constants, given as the float32 values the kernels use (the
    oracle widens them exactly)."""
    sigma: float = float(np.float32(1.0 / np.sqrt(2.0)))   # screen-space low-pass, px
    det_eps: float = float(np.float32(1e-6))               # |det M| threshold, px^2
    alpha_min: float = float(np.float32(1.0 / 255.0))
    alpha_max: float = float(np.float32(0.99))
    t_min: float = float(np.float32(1e-4))

    def record(self) -> np.ndarray:
        return np.array([self.sigma, self.det_eps, self.alpha_min, self.alpha_max, self.t_min],
                        dtype=np.float64)


def camera_record(cam, dF=None, color=None) -> np.ndarray:
    """Flat float64 camera record from a ``scenegen.Camera`` (values widened exactly).
    ``dF`` / ``color`` override the camera's own delta / colour matrix."""
    r = np.zeros(C_NUM, dtype=np.float64)
    r[C_F:C_F + 8] = np.asarray(cam.F_xy, dtype=np.float32).astype(np.float64).ravel()
    d = cam.dF_xy if dF is None else dF
    r[C_DF:C_DF + 8] = np.asarray(d, dtype=np.float32).astype(np.float64).ravel()
    r[C_MAXALT] = float(np.float32(cam.max_alt))
    r[C_W], r[C_H] = cam.width, cam.height
    col = cam.color if color is None else color
    r[C_COLOR:C_COLOR + 12] = np.asarray(col, dtype=np.float32).astype(np.float64).ravel()
    r[C_PHI] = float(np.float32(cam.sun_phi))
    r[C_THETA] = float(np.float32(cam.sun_theta))
    r[C_SW], r[C_SH] = cam.shadow_w, cam.shadow_h
    r[C_SSCALE] = float(np.float32(cam.shadow_scale))
    return r


class SceneF64:
    """A scene's splat arrays widened to float64 (planar [C][N])."""

    def __init__(self, means, scales, quats, opacity, rgb):
        self.means = _d(means)
        self.scales = _d(scales)
        self.quats = _d(quats)
        self.opacity = _d(opacity)
        self.rgb = _d(rgb)
        self.n = int(self.means.shape[1])

    @classmethod
    def of(cls, scene):
        return cls(scene.means, scene.scales, scene.quats, scene.opacity, scene.rgb)

    def args(self):
        return [self.n, _ptr(self.means), _ptr(self.scales), _ptr(self.quats),
                _ptr(self.opacity), _ptr(self.rgb)]


def _crop(cam, sun, crop):
    W, H = (cam.shadow_w, cam.shadow_h) if sun else (cam.width, cam.height)
    if crop is None:
        return 0, 0, W, H
    x0, y0, w, h = crop
    assert 0 <= x0 and 0 <= y0 and x0 + w <= W and y0 + h <= H
    return int(x0), int(y0), int(w), int(h)


def set_threads(n: int) -> None:
    lib().ora_set_threads(int(n))


def num_threads() -> int:
    return int(lib().ora_num_threads())


def camera(cam, sun=False, dF=None):
    B = np.zeros(6); b = np.zeros(2); vs = np.zeros(3); wh = np.zeros(2, dtype=np.int32)
    rec = camera_record(cam, dF=dF)
    lib().ora_camera(_ptr(rec), int(sun), _ptr(B), _ptr(b), _ptr(vs), _ptr(wh))
    return B.reshape(2, 3), b, vs, (int(wh[0]), int(wh[1]))


PROJ_FIELDS = ["M00", "M01", "M10", "M11", "det", "Q00", "Q01", "Q10", "Q11", "q0", "q1",
               "cx", "cy", "zc", "dzdu", "dzdv", "nx", "ny", "nz", "r2", "ex", "ey", "deg", "culled"]


def project(sc: SceneF64, cam, sun=False, opts: Opts = Opts(), dF=None):
    out = np.zeros((sc.n, 24))
    rec = camera_record(cam, dF=dF)
    o = opts.record()
    lib().ora_project(*sc.args(), _ptr(rec), int(sun), _ptr(o), _ptr(out))
    return {f: out[:, i] for i, f in enumerate(PROJ_FIELDS)}


def order(sc: SceneF64) -> np.ndarray:
    out = np.zeros(sc.n, dtype=np.int64)
    lib().ora_order(sc.n, _ptr(sc.means), _ptr(out))
    return out


def render(sc: SceneF64, cam, sun=False, opts: Opts = Opts(), crop=None, brute=False,
           dF=None, color=None):
    """Forward render of a view (or its sun view).  Returns a dict of float64 planes:
    rgb (3,h,w), depth, normal (3,h,w), alpha, distort (the distortion of the blending weights
    along the ray, Supp. B), T, margin_fwd, margin_bwd and int32 ncontrib / terminated.
    ``color`` is the 3x4 [C|c] (identity for sun views)."""
    x0, y0, w, h = _crop(cam, sun, crop)
    rec = camera_record(cam, dF=dF, color=color)
    col = rec[C_COLOR:C_COLOR + 12].copy()
    o = opts.record()
    out = dict(rgb=np.zeros((3, h, w)), depth=np.zeros((h, w)), normal=np.zeros((3, h, w)),
               alpha=np.zeros((h, w)), T=np.zeros((h, w)), margin_fwd=np.zeros((h, w)),
               margin_bwd=np.zeros((h, w)), ncontrib=np.zeros((h, w), np.int32),
               terminated=np.zeros((h, w), np.int32), distort=np.zeros((h, w)))
    lib().ora_render(*sc.args(), _ptr(rec), int(sun), _ptr(col), _ptr(o), x0, y0, w, h, int(brute),
                     _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["normal"]), _ptr(out["alpha"]),
                     _ptr(out["T"]), _ptr(out["margin_fwd"]), _ptr(out["margin_bwd"]),
                     _ptr(out["ncontrib"]), _ptr(out["terminated"]), _ptr(out["distort"]))
    return out


def render_dual(sc: SceneF64, cam, tangents: dict, sun=False, opts: Opts = Opts(), crop=None,
                brute=False, dF=None, color=None):
    """Forward-mode derivative of the rendered planes along ``tangents`` (keys: means,
    scales, quats, opacity, rgb, dF, color; missing = 0)."""
    x0, y0, w, h = _crop(cam, sun, crop)
    rec = camera_record(cam, dF=dF, color=color)
    col = rec[C_COLOR:C_COLOR + 12].copy()
    o = opts.record()
    t = {k: (None if tangents.get(k) is None else _d(tangents[k]))
         for k in ("means", "scales", "quats", "opacity", "rgb", "dF", "color")}
    out = dict(rgb=np.zeros((3, h, w)), depth=np.zeros((h, w)), normal=np.zeros((3, h, w)),
               alpha=np.zeros((h, w)), distort=np.zeros((h, w)))
    lib().ora_render_dual(*sc.args(), _ptr(rec), int(sun), _ptr(col), _ptr(o), x0, y0, w, h,
                          int(brute), _ptr(t["means"]), _ptr(t["scales"]), _ptr(t["quats"]),
                          _ptr(t["opacity"]), _ptr(t["rgb"]), _ptr(t["dF"]), _ptr(t["color"]),
                          _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["normal"]),
                          _ptr(out["alpha"]), _ptr(out["distort"]))
    return out


def backward(sc: SceneF64, cam, upstream: dict, sun=False, opts: Opts = Opts(), crop=None,
             brute=False, dF=None, color=None):
    """Reverse-mode gradients of sum(upstream * planes) for the crop.  ``upstream`` keys:
    rgb (3,h,w), depth (h,w), normal (3,h,w), alpha (h,w), distort (h,w); missing = 0."""
    x0, y0, w, h = _crop(cam, sun, crop)
    rec = camera_record(cam, dF=dF, color=color)
    col = rec[C_COLOR:C_COLOR + 12].copy()
    o = opts.record()
    g = {k: (None if upstream.get(k) is None else _d(upstream[k]))
         for k in ("rgb", "depth", "normal", "alpha", "distort")}
    n = sc.n
    out = dict(means=np.zeros((3, n)), scales=np.zeros((2, n)), quats=np.zeros((4, n)),
               opacity=np.zeros(n), rgb=np.zeros((3, n)), dF=np.zeros(8), color=np.zeros(12))
    lib().ora_backward(*sc.args(), _ptr(rec), int(sun), _ptr(col), _ptr(o), x0, y0, w, h,
                       int(brute), _ptr(g["rgb"]), _ptr(g["depth"]), _ptr(g["normal"]),
                       _ptr(g["alpha"]), _ptr(g["distort"]), _ptr(out["means"]), _ptr(out["scales"]),
                       _ptr(out["quats"]), _ptr(out["opacity"]), _ptr(out["rgb"]),
                       _ptr(out["dF"]), _ptr(out["color"]))
    out["dF"] = out["dF"].reshape(2, 4)
    out["color"] = out["color"].reshape(3, 4)
    return out
