"""Reading and writing the golden fixtures (JSON text) of this folder: splats, cameras and
expected values.  Plain serialisation; no rasterizer arithmetic here."""
from __future__ import annotations

import json
import os

import numpy as np

import scenegen

HERE = os.path.dirname(os.path.abspath(__file__))


def f32(x):
    """Values rounded to float32, written as the shortest decimals that read back as the same
    float32 values (both paths read float32 inputs)."""
    a = np.asarray(x, np.float32)
    if a.ndim == 0:
        return float(str(a[()]))  # numpy prints the shortest float32 round-trip digits
    return [f32(v) for v in a]


def g12(x):
    """Expected values to 12 significant digits (far below every tolerance that reads them)."""
    a = np.asarray(x, np.float64)
    if a.ndim == 0:
        return float(f"{float(a):.12g}")
    return [g12(v) for v in a]


def splats_json(means, scales, quats, opacity, rgb) -> dict:
    return dict(means=f32(np.reshape(means, (3, -1))), scales=f32(np.reshape(scales, (2, -1))),
                quats=f32(np.reshape(quats, (4, -1))), opacity=f32(np.reshape(opacity, (-1,))),
                rgb=f32(np.reshape(rgb, (3, -1))))


def camera_json(cam: scenegen.Camera) -> dict:
    return dict(F_xy=f32(cam.F_xy), dF_xy=f32(cam.dF_xy), max_alt=f32(cam.max_alt),
                width=int(cam.width), height=int(cam.height), color=f32(cam.color),
                sun_phi=f32(cam.sun_phi), sun_theta=f32(cam.sun_theta), shadow_w=int(cam.shadow_w),
                shadow_h=int(cam.shadow_h), shadow_scale=f32(cam.shadow_scale))


def camera_of(d: dict) -> scenegen.Camera:
    a = lambda k: np.asarray(d[k], np.float32)
    s = lambda k: float(np.float32(d[k]))
    return scenegen.Camera(F_xy=a("F_xy"), dF_xy=a("dF_xy"), max_alt=s("max_alt"),
                           width=int(d["width"]), height=int(d["height"]), color=a("color"),
                           sun_phi=s("sun_phi"), sun_theta=s("sun_theta"),
                           shadow_w=int(d["shadow_w"]), shadow_h=int(d["shadow_h"]),
                           shadow_scale=s("shadow_scale"))


def scene_of(case: dict) -> scenegen.Scene:
    s = case["splats"]
    a = lambda k: np.asarray(s[k], np.float32)
    return scenegen.Scene(means=a("means"), scales=a("scales"), quats=a("quats"), opacity=a("opacity"),
                          rgb=a("rgb"), cameras=[camera_of(case["camera"])], scale_m=1.0,
                          name=case["name"])


def load(name: str) -> dict:
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def _text(obj, ind: str) -> str:
    """JSON with one key per line and every list of numbers on one line."""
    if isinstance(obj, dict):
        inner = ind + " "
        items = [f"{inner}{json.dumps(k)}: {_text(v, inner)}" for k, v in obj.items()]
        return "{\n" + ",\n".join(items) + "\n" + ind + "}"
    if isinstance(obj, list) and any(isinstance(v, dict) for v in obj):
        inner = ind + " "
        return "[\n" + ",\n".join(inner + _text(v, inner) for v in obj) + "\n" + ind + "]"
    return json.dumps(obj)


def dump(obj: dict, name: str) -> None:
    with open(os.path.join(HERE, name), "w") as f:
        f.write(_text(obj, "") + "\n")


def upstream(width: int, height: int, sun: bool) -> dict:
    """The fixed upstream gradients of the stored-scene fixture: smooth functions of the pixel
    (column x, row y, channel c), stated here and in the fixture."""
    y, x = np.mgrid[0:height, 0:width].astype(np.float64)
    c = np.arange(3, dtype=np.float64)[:, None, None]
    u = dict(depth=np.cos(0.29 * x - 0.53 * y), alpha=np.cos(0.17 * x + 0.71 * y + 0.5))
    if not sun:
        u.update(rgb=np.sin(0.37 * x + 0.61 * y + 1.3 * c), normal=np.sin(0.41 * x + 0.23 * y - 0.7 * c),
                 distort=np.sin(0.5 * x - 0.3 * y))
    # the kernels read float32 upstream planes: both sides take the rounded values
    return {k: v.astype(np.float32).astype(np.float64) for k, v in u.items()}


UPSTREAM_TEXT = ("rgb[c,y,x] = sin(0.37x + 0.61y + 1.3c), depth = cos(0.29x - 0.53y), "
                 "normal[c] = sin(0.41x + 0.23y - 0.7c), alpha = cos(0.17x + 0.71y + 0.5), "
                 "distort = sin(0.5x - 0.3y) (main view); depth and alpha alike on the sun view; "
                 "rounded to float32")
