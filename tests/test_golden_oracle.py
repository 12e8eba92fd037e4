"""The oracle against the golden fixtures of tests/golden: values that follow from the paper's
equations by hand (closed_forms.json, written with `math` alone), and the oracle's own stored
planes and gradients of a small seeded scene (oracle_scene.json), which pin its arithmetic
against unintended change."""
import numpy as np
import pytest

import oracle
from tests.golden import fixtures as FX
from tests.golden import write_closed_forms

CLOSED = FX.load("closed_forms.json")
SCENE = FX.load("oracle_scene.json")


def _close(got, want, rtol, name):
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    tol = rtol * np.maximum(np.abs(want), 1e-3 * max(float(np.abs(want).max()), 1e-30))
    bad = np.abs(got - want) > tol
    assert not bad.any(), f"{name}: got {got[bad][:4]}, want {want[bad][:4]}"


def _render_case(case):
    sc = FX.scene_of(case)
    cam = sc.cameras[0]
    sun = case["view"] == "sun"
    return sc, cam, oracle.render(oracle.SceneF64.of(sc), cam, sun=sun, color=None if sun else cam.color)


def _at(planes, key, pixels):
    a = planes[key]
    return np.array([a[..., j, i] for (i, j) in pixels])


@pytest.mark.parametrize("name", [c["name"] for c in CLOSED["cases"]])
def test_oracle_matches_the_closed_forms(name):
    case = next(c for c in CLOSED["cases"] if c["name"] == name)
    _, _, out = _render_case(case)
    for key, want in case["expected"].items():
        _close(_at(out, key, case["pixels"]), want, 1e-10, f"{name}.{key}")
    # the zero-alpha pixels of the cases are exactly empty
    for (i, j), a in zip(case["pixels"], case["expected"].get("alpha", [])):
        if a == 0.0:
            assert out["alpha"][j, i] == 0.0


def test_oracle_gradient_matches_the_closed_form():
    case = next(c for c in CLOSED["cases"] if "grad" in c)
    sc, cam, out = _render_case(case)
    g = case["grad"]
    i, j = g["pixel"]
    ups = dict(alpha=np.zeros((cam.height, cam.width)), rgb=np.zeros((3, cam.height, cam.width)))
    ups["alpha"][j, i] = g["d_alpha"]
    ups["rgb"][:, j, i] = g["d_rgb"]
    r = oracle.backward(oracle.SceneF64.of(sc), cam, ups, color=cam.color)
    for key, want in g["expected"].items():
        got = np.asarray(r[key]).reshape(-1)
        want = np.asarray(want)
        scale = float(np.abs(want).max())
        assert np.abs(got - want).max() <= 1e-9 * scale, (key, got, want)


def test_closed_forms_file_is_what_its_writer_writes():
    fresh = write_closed_forms.build()
    assert [c["name"] for c in fresh["cases"]] == [c["name"] for c in CLOSED["cases"]]
    for a, b in zip(fresh["cases"], CLOSED["cases"]):
        assert a["pixels"] == b["pixels"] and a["splats"] == b["splats"] and a["camera"] == b["camera"]
        for key in a["expected"]:
            np.testing.assert_array_equal(np.asarray(a["expected"][key]), np.asarray(b["expected"][key]))


def test_oracle_reproduces_its_stored_scene():
    sc = FX.scene_of(SCENE)
    cam = sc.cameras[0]
    s64 = oracle.SceneF64.of(sc)
    main = oracle.render(s64, cam, color=cam.color)
    sun = oracle.render(s64, cam, sun=True)
    for key, want in SCENE["main"].items():
        _close(main[key], want, 1e-9, f"main.{key}")
    for key, want in SCENE["sun"].items():
        _close(sun[key], want, 1e-9, f"sun.{key}")
    # every decision keeps its margin (the reason the seed was chosen)
    for o in (main, sun):
        assert o["margin_fwd"].min() >= 1e-4 and o["margin_bwd"].min() >= 1e-4
    gm = oracle.backward(s64, cam, FX.upstream(cam.width, cam.height, False), color=cam.color)
    gs = oracle.backward(s64, cam, FX.upstream(cam.shadow_w, cam.shadow_h, True), sun=True)
    for key in SCENE["grad_main"]:
        _close(gm[key], SCENE["grad_main"][key], 1e-9, f"grad_main.{key}")
        _close(gs[key], SCENE["grad_sun"][key], 1e-9, f"grad_sun.{key}")
