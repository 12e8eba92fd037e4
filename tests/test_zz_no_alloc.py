"""The allocation-free entry point (for callers that cannot call cudaMalloc, e.g. under a device
memory budget fixed at start-up, or plug-ins given a stream but no allocator): its forward render
must equal the workspace path's, call after call, although every call reuses the library's
static scratch.
Collected last on purpose."""
import ctypes

import pytest
import torch

import scenegen
from paper_2606_28581_gb300 import _lib as L
from paper_2606_28581_gb300.frame import Outputs
from tests.gpu_util import FWD_TOL, DeviceScene, run_forward

pytestmark = pytest.mark.gpu


def test_noalloc_forward_matches_workspace_path_twice():
    scene = scenegen.make_scene(n=3000, extent_m=80.0, seed=31,
                                views=[dict(width=100, height=75, off_nadir=20.0, delta=True, color_noise=0.02)])
    ds = DeviceScene(scene)
    frame, ref = run_forward(ds)  # the workspace-based entry points
    cams = L.make_cameras(scene.cameras)
    opts = L.default_opts()
    for call in range(2):
        out = Outputs(frame.targets, "cuda")
        for plane in (out.rgb[0], out.depth[0], out.normal[0], out.alpha[0]):
            plane.fill_(float("nan"))
        st, needed = L.render_fwd_noalloc(ds.splats, cams, ds.dF, ds.color, opts, out.io_array())
        torch.cuda.synchronize()
        assert st == L.SS_OK and needed == frame.needed, (call, st, needed)
        for name in ("rgb", "depth", "normal", "alpha", "T_final"):
            a = getattr(ref, name)[0]
            b = getattr(out, name)[0]
            assert torch.isfinite(b).all(), (call, name)
            assert float((a - b).abs().max()) <= FWD_TOL, (call, name)
        assert torch.equal(ref.last[0], out.last[0])


def test_noalloc_rejects_a_scene_beyond_its_scratch():
    n = 1 << 20  # 1M splats need more workspace than the 64 MiB array holds
    assert L.noalloc_scratch_bytes() == 64 << 20
    z = torch.zeros(3, n, device="cuda")
    s = L.make_splats(z, z[:2], torch.zeros(4, n, device="cuda"), z[:1], z, n)
    cam = scenegen.make_scene(n=8, extent_m=10.0, views=[dict(width=64, height=64)]).cameras
    io = Outputs([type("T", (), dict(sun=False, width=64, height=64))()], "cuda").io_array()
    st = L.load().ss_render_fwd_noalloc(ctypes.byref(s), L.make_cameras(cam), None, None,
                                        ctypes.byref(L.default_opts()), io, None, None)
    assert st == L.SS_ERR_INVALID_ARG
