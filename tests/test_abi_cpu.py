"""Host-only checks of the C ABI: the library builds for sm_103a, loads, and exports every
entry point that include/satsplat.h declares; host-side helpers need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_28581_gb300.build import build
    build()
    from paper_2606_28581_gb300 import _lib as L
    return L.load()


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "satsplat.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(ss_[a-z_]+)\s*\(", hdr)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("ss_project_splats", "ss_bin_and_sort", "ss_rasterize_fwd", "ss_rasterize_bwd", "ss_shadow_depth"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2606_28581_gb300 import _lib as L
    assert sorted(L.EXPORTS) == declared_symbols()


def test_default_opts_and_status_strings(lib):
    from paper_2606_28581_gb300 import _lib as L
    o = L.default_opts()
    assert (o.tile_w, o.tile_h, o.batch, o.persistent, o.pixels_per_thread, o.count_pairs) == (16, 16, 256, 0, 4, 0)
    assert abs(o.alpha_min - 1 / 255) < 1e-9 and abs(o.alpha_max - 0.99) < 1e-7 and abs(o.t_min - 1e-4) < 1e-9
    assert L.status_string(L.SS_ERR_CAPACITY) == "intersection capacity exceeded"


def test_staging_batches_fit_the_kernels_slot_encoding(lib):
    """The rasterizer's staged batches: whole 32-record chunks (the candidate masks) and at most
    256 records (a candidate's slot is one byte)."""
    from paper_2606_28581_gb300 import _lib as L
    fwd, bwd = L.staging_batches()
    for b in (fwd, bwd):
        assert 32 <= b <= 256 and b % 32 == 0, b


def test_workspace_size_validates_on_the_host(lib):
    import scenegen
    from paper_2606_28581_gb300 import _lib as L
    sc = scenegen.workload("small")
    cams = L.make_cameras(sc.cameras)
    s = L.ss_splats()
    s.means = s.scales = s.quats = s.opacity = s.rgb = 4096  # never dereferenced on the host
    s.n, s.n_pad, s.dtype = sc.n, sc.n, L.SS_F32
    o = L.default_opts()
    size = L.workspace_size(s, cams, 1, L.SS_PASS_MAIN | L.SS_PASS_SUN, o, 1 << 20)
    assert size > 2 * sc.n * (48 + 32 + 8 + 64)
    out = ctypes.c_size_t(0)
    for bad in (L.default_opts(batch=100), L.default_opts(batch=128), L.default_opts(pixels_per_thread=2),
                L.default_opts(tile_w=32, tile_h=32), L.default_opts(subblock_cull=2),
                L.default_opts(count_pairs=2)):
        assert lib.ss_workspace_size(ctypes.byref(s), cams, 1, 1, ctypes.byref(bad), 1 << 20,
                                     ctypes.byref(out)) == L.SS_ERR_INVALID_ARG
    assert lib.ss_workspace_size(ctypes.byref(s), cams, 1, 1, ctypes.byref(bad), 1 << 20,
                                 ctypes.byref(out)) == L.SS_ERR_INVALID_ARG
    s.n_pad = sc.n + 1
    assert lib.ss_workspace_size(ctypes.byref(s), cams, 1, 1, ctypes.byref(o), 1 << 20,
                                 ctypes.byref(out)) == L.SS_ERR_INVALID_ARG
    s.n_pad = sc.n
    s.means = 4100  # not 16-byte aligned
    assert lib.ss_workspace_size(ctypes.byref(s), cams, 1, 1, ctypes.byref(o), 1 << 20,
                                 ctypes.byref(out)) == L.SS_ERR_INVALID_ARG


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2606_28581_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
