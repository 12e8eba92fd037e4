"""Geometry-aware initialisation (Sec. 3.4) on the GPU against the FP64 oracle, through the C ABI:
the sampled pixels (exact integer decisions), the jittered centres, the Gram-Schmidt rotation,
the colour and the kNN scales."""
import numpy as np
import pytest
import torch

import scenegen
from oracle import init as I
from oracle import optim as O
from paper_2606_28581_gb300 import _lib as L
from paper_2606_28581_gb300.frame import n_pad_of
from tests.gpu_util import to_np

pytestmark = pytest.mark.gpu


def _run(dsm, n, dtype, seed, k=3):
    Z = torch.from_numpy(dsm.height).cuda()
    rgb = torch.from_numpy(dsm.rgb).cuda()
    d = L.make_dsm(Z, rgb, dsm.x0, dsm.y0, dsm.gsd)
    n_pad = n_pad_of(n)
    z = lambda c: torch.zeros(c, n_pad, device="cuda", dtype=dtype)
    st = dict(means=z(3), scales=z(2), quats=z(4), opacity=z(1), rgb=z(3))
    out = L.make_splats(st["means"], st["scales"], st["quats"], st["opacity"], st["rgb"], n)
    ws = torch.empty(L.init_workspace_size(d, n), dtype=torch.uint8, device="cuda")
    L.dsm_init(d, L.default_init_opts(seed=seed, knn_k=k), out, ws)
    torch.cuda.synchronize()
    return {kk: to_np(t)[:, :n] for kk, t in st.items()}


def _compare(g, ora, sel, dtype):
    """Positions to FP32 rounding (6e-7 absolute: the sums cancel near zero), plus with BF16
    storage one unit in the last place (at most 2^-7 of the value: the FP32 value may round the
    other way); a different pixel would be a whole pixel away."""
    bf16 = dtype == torch.bfloat16
    gm = g["means"][:, sel]
    bound = 6e-7 + (2.0 ** -7 * np.abs(ora["means"]) if bf16 else 0.0)
    assert np.all(np.abs(gm - ora["means"]) <= bound), np.abs(gm - ora["means"]).max()
    R = O.rotation(g["quats"][:, sel])
    assert np.abs(R - ora["R"]).max() <= (3e-2 if bf16 else 2e-5)
    rgb = ora["rgb"].astype(np.float32)
    rgb = scenegen.to_bf16_exact(rgb) if bf16 else rgb
    np.testing.assert_array_equal(g["rgb"][:, sel], rgb.astype(np.float64))
    np.testing.assert_allclose(g["scales"][:, sel], ora["scales"], rtol=1e-2 if bf16 else 2e-4)
    assert np.all(g["scales"][0] == g["scales"][1])
    op = scenegen.to_bf16_exact(np.float32(0.1)) if bf16 else np.float32(0.1)
    assert np.all(g["opacity"] == np.float64(op))


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_dsm_init_matches_oracle(dtype):
    dsm = scenegen.make_dsm(size_px=200, extent_m=100.0, seed=5)
    n = 20011
    g = _run(dsm, n, dtype, seed=17)
    ora = I.init_splats(dsm, n, seed=17)
    _compare(g, ora, np.arange(n), dtype)
    # facades are sampled more densely than flat ground, per pixel
    w = I.weights(dsm)
    assert w.max() > 10 * np.median(w)


def test_dsm_init_full_size_1M_samples():
    """A 2048 x 2048 DSM of 1 km^2 at 0.5 m and 1M samples; every sample's pixel and centre, and
    the rotation, colour and kNN scale of 20000 of them, against the oracle."""
    dsm = scenegen.make_dsm(size_px=2048, extent_m=1000.0, seed=6)
    n = 1_000_000
    g = _run(dsm, n, torch.float32, seed=3)
    sel = np.sort(np.random.default_rng(0).choice(n, 20000, replace=False))
    ora = I.init_splats(dsm, n, seed=3, index=sel)
    _compare(g, ora, sel, torch.float32)
    # every centre (the drawn pixel of every sample)
    w = I.weights(dsm)
    pix, u, v = I.draw_pixels(w, n, 3)
    W = dsm.height.shape[1]
    gx = float(np.float32(dsm.x0)) + (pix % W + u) * float(np.float32(dsm.gsd))
    assert np.abs(g["means"][0] - gx).max() <= 6e-7


def test_dsm_init_rejects_bad_arguments():
    dsm = scenegen.make_dsm(size_px=16, extent_m=8.0, seed=1)
    Z = torch.from_numpy(dsm.height).cuda()
    d = L.make_dsm(Z, None, dsm.x0, dsm.y0, dsm.gsd)
    st = torch.zeros(3, 8, device="cuda")
    out = L.make_splats(st, st[:2], torch.zeros(4, 8, device="cuda"), st[:1], st, 3)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(L.SatSplatError):  # n must exceed knn_k
        L.dsm_init(d, L.default_init_opts(knn_k=3), out, ws)
    with pytest.raises(L.SatSplatError):
        L.dsm_init(d, L.default_init_opts(knn_k=9), out, ws)
    bad = L.make_dsm(Z, None, dsm.x0, dsm.y0, -1.0)
    with pytest.raises(L.SatSplatError):
        L.init_workspace_size(bad, 100)
