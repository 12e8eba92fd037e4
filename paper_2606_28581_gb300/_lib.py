"""ctypes binding of ``include/satsplat.h`` (argument marshalling only).

Every function here has the name of the C entry point without the ``ss_``
prefix and forwards to it.  Tensors are passed as raw device pointers; the
CUDA stream is torch's current stream unless one is given.  Loading fails
loudly when the compiled library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsatsplat.so")

SS_OK, SS_ERR_INVALID_ARG, SS_ERR_CAPACITY, SS_ERR_CUDA, SS_ERR_TIMEOUT, SS_ERR_NONFINITE = range(6)
SS_F32, SS_BF16 = 0, 1
SS_PASS_MAIN, SS_PASS_SUN = 1, 2

P = ctypes.c_void_p


class ss_splats(ctypes.Structure):
    _fields_ = [("means", P), ("scales", P), ("quats", P), ("opacity", P), ("rgb", P),
                ("n", ctypes.c_int64), ("n_pad", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ss_camera(ctypes.Structure):
    _fields_ = [("F_xy", (ctypes.c_float * 4) * 2), ("max_alt", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("sun_phi", ctypes.c_float), ("sun_theta", ctypes.c_float),
                ("shadow_w", ctypes.c_int32), ("shadow_h", ctypes.c_int32),
                ("shadow_scale", ctypes.c_float)]


class ss_raster_opts(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("sigma_px", ctypes.c_float),
                ("det_eps", ctypes.c_float), ("alpha_min", ctypes.c_float),
                ("alpha_max", ctypes.c_float), ("t_min", ctypes.c_float),
                ("pixels_per_thread", ctypes.c_int32), ("subblock_cull", ctypes.c_int32),
                ("count_pairs", ctypes.c_int32)]


class ss_target_io(ctypes.Structure):
    _fields_ = [("rgb", P), ("depth", P), ("normal", P), ("alpha", P), ("T_final", P), ("last", P),
                ("d_rgb", P), ("d_depth", P), ("d_normal", P), ("d_alpha", P), ("distort", P),
                ("d_distort", P)]


class ss_shade_opts(ctypes.Structure):
    _fields_ = [("esm_k", ctypes.c_float), ("esm_bias", ctypes.c_float), ("alpha_eps", ctypes.c_float)]


class ss_shade_io(ctypes.Structure):
    _fields_ = [("rgb", P), ("depth", P), ("alpha", P), ("sun_depth", P), ("sun_alpha", P), ("image", P),
                ("vis", P), ("d_image", P), ("d_rgb", P), ("d_depth", P), ("d_alpha", P),
                ("d_sun_depth", P), ("d_sun_alpha", P)]


class ss_dnormal_io(ctypes.Structure):
    _fields_ = [("depth", P), ("alpha", P), ("normal", P), ("d_normal", P), ("d_depth", P), ("d_alpha", P)]


class ss_splat_grads(ctypes.Structure):
    _fields_ = [("means", P), ("scales", P), ("quats", P), ("opacity", P), ("rgb", P),
                ("n_pad", ctypes.c_int64)]


class ss_splat_params(ctypes.Structure):
    _fields_ = [("means", P), ("log_scales", P), ("quats", P), ("logit_opacity", P), ("rgb", P),
                ("n_pad", ctypes.c_int64)]


class ss_adam_opts(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("lr_means", "lr_scales", "lr_quats", "lr_opacity", "lr_rgb", "beta1",
                                               "beta2", "eps", "noise_lr", "noise_k", "noise_t")] + \
               [("step", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class ss_dsm(ctypes.Structure):
    _fields_ = [("heights", P), ("rgb", P), ("width", ctypes.c_int32), ("height_px", ctypes.c_int32),
                ("x0", ctypes.c_float), ("y0", ctypes.c_float), ("gsd", ctypes.c_float)]


class ss_init_opts(ctypes.Structure):
    _fields_ = [("knn_k", ctypes.c_int32), ("opacity", ctypes.c_float), ("seed", ctypes.c_uint64)]


class ss_mcmc_opts(ctypes.Structure):
    _fields_ = [("min_opacity", ctypes.c_float), ("growth", ctypes.c_float), ("n_max", ctypes.c_int32),
                ("step", ctypes.c_int32), ("seed", ctypes.c_uint64)]


EXPORTS = ["ss_default_opts", "ss_status_string", "ss_staging_batches", "ss_workspace_size", "ss_project_splats",
           "ss_bin_and_sort", "ss_rasterize_fwd", "ss_rasterize_bwd", "ss_project_bwd", "ss_shadow_depth",
           "ss_frame_status", "ss_device_info", "ss_kernel_launches", "ss_render_fwd_noalloc",
           "ss_noalloc_scratch_bytes", "ss_default_shade_opts", "ss_shade_fwd", "ss_shade_bwd",
           "ss_depth_normal_fwd", "ss_depth_normal_bwd", "ss_default_adam_opts", "ss_adam_step", "ss_adam_flat",
           "ss_default_mcmc_opts", "ss_mcmc_workspace_size", "ss_mcmc_relocate", "ss_default_init_opts",
           "ss_init_workspace_size", "ss_dsm_init"]

_lock = threading.Lock()
_lib = None


class SatSplatError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


def load(path: Optional[str] = None):
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"CUDA library not built: {p} is missing (run paper_2606_28581_gb300.build.build())")
        L = ctypes.CDLL(p)
        I32, I64, SZ = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        PS, PC, PO = ctypes.POINTER(ss_splats), ctypes.POINTER(ss_camera), ctypes.POINTER(ss_raster_opts)
        PIO, PG = ctypes.POINTER(ss_target_io), ctypes.POINTER(ss_splat_grads)
        L.ss_default_opts.argtypes = [PO]
        L.ss_default_opts.restype = None
        L.ss_status_string.argtypes = [ctypes.c_int]
        L.ss_status_string.restype = ctypes.c_char_p
        L.ss_staging_batches.argtypes = [ctypes.POINTER(I32), ctypes.POINTER(I32)]
        L.ss_staging_batches.restype = None
        L.ss_workspace_size.argtypes = [PS, PC, I32, I32, PO, I64, ctypes.POINTER(SZ)]
        L.ss_project_splats.argtypes = [PS, PC, I32, I32, P, P, PO, P, SZ, I64, P]
        L.ss_bin_and_sort.argtypes = [PS, PC, I32, I32, PO, P, SZ, I64, ctypes.POINTER(I64), P]
        L.ss_rasterize_fwd.argtypes = [PS, PC, I32, I32, PO, PIO, P, SZ, I64, P]
        L.ss_rasterize_bwd.argtypes = [PS, PC, I32, I32, PO, PIO, PG, P, P, P, SZ, I64, P]
        L.ss_project_bwd.argtypes = [PS, PC, I32, I32, PO, PG, P, P, P, SZ, I64, P]
        L.ss_shadow_depth.argtypes = [PS, PC, I32, P, PO, PIO, P, SZ, I64, ctypes.POINTER(I64), P]
        L.ss_frame_status.argtypes = [P, SZ, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64),
                                      ctypes.POINTER(I32), P]
        L.ss_device_info.argtypes = [ctypes.POINTER(I32), ctypes.POINTER(I32)]
        L.ss_device_info.restype = I32
        L.ss_render_fwd_noalloc.argtypes = [PS, PC, P, P, PO, PIO, ctypes.POINTER(I64), P]
        L.ss_noalloc_scratch_bytes.argtypes = []
        L.ss_noalloc_scratch_bytes.restype = SZ
        L.ss_kernel_launches.argtypes = []
        L.ss_kernel_launches.restype = I64
        PSO, PSI = ctypes.POINTER(ss_shade_opts), ctypes.POINTER(ss_shade_io)
        L.ss_default_shade_opts.argtypes = [PSO]
        L.ss_default_shade_opts.restype = None
        L.ss_shade_fwd.argtypes = [PC, I32, P, P, PSO, PSI, P]
        L.ss_shade_bwd.argtypes = [PC, I32, P, P, PSO, PSI, P, P, P]
        PNI = ctypes.POINTER(ss_dnormal_io)
        L.ss_depth_normal_fwd.argtypes = [PC, I32, P, ctypes.c_float, PNI, P]
        L.ss_depth_normal_bwd.argtypes = [PC, I32, P, ctypes.c_float, PNI, P, P]
        PPA, PAO, PMO = ctypes.POINTER(ss_splat_params), ctypes.POINTER(ss_adam_opts), ctypes.POINTER(ss_mcmc_opts)
        L.ss_default_adam_opts.argtypes = [PAO]
        L.ss_default_adam_opts.restype = None
        L.ss_adam_step.argtypes = [PPA, PPA, PPA, PG, PS, PAO, P]
        L.ss_adam_flat.argtypes = [P, P, P, P, I64, ctypes.c_float, PAO, P]
        L.ss_default_mcmc_opts.argtypes = [PMO]
        L.ss_default_mcmc_opts.restype = None
        L.ss_mcmc_workspace_size.argtypes = [I64, ctypes.POINTER(SZ)]
        L.ss_mcmc_relocate.argtypes = [PPA, PPA, PPA, PS, I64, PMO, P, SZ, ctypes.POINTER(I64), P, P]
        PD, PIN = ctypes.POINTER(ss_dsm), ctypes.POINTER(ss_init_opts)
        L.ss_default_init_opts.argtypes = [PIN]
        L.ss_default_init_opts.restype = None
        L.ss_init_workspace_size.argtypes = [PD, I64, ctypes.POINTER(SZ)]
        L.ss_dsm_init.argtypes = [PD, PIN, PS, P, SZ, P]
        for name in EXPORTS:
            if name not in ("ss_default_opts", "ss_status_string", "ss_staging_batches", "ss_device_info",
                            "ss_kernel_launches",
                            "ss_noalloc_scratch_bytes", "ss_default_shade_opts", "ss_default_adam_opts",
                            "ss_default_mcmc_opts", "ss_default_init_opts"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def staging_batches() -> tuple:
    """Records per staged batch of the forward and the backward rasterizer kernels."""
    f, b = ctypes.c_int32(0), ctypes.c_int32(0)
    load().ss_staging_batches(ctypes.byref(f), ctypes.byref(b))
    return f.value, b.value


def status_string(status: int) -> str:
    try:
        return load().ss_status_string(int(status)).decode()
    except Exception:  # pragma: no cover - only used in error paths
        return "status"


def _check(status: int, where: str, allow=()):
    if status != SS_OK and status not in allow:
        raise SatSplatError(status, where)
    return status


# ------------------------------------------------------------------------------ marshalling
def ptr(t) -> Optional[int]:
    if t is None:
        return None
    return int(t.data_ptr())


def stream_ptr(stream=None) -> Optional[int]:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream) or None


def default_opts(**overrides) -> ss_raster_opts:
    o = ss_raster_opts()
    load().ss_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def make_cameras(cams: Sequence) -> ctypes.Array:
    """Array of ss_camera from objects with F_xy (2x4), max_alt, width, height, sun_phi,
    sun_theta, shadow_w, shadow_h, shadow_scale attributes."""
    arr = (ss_camera * len(cams))()
    for i, c in enumerate(cams):
        F = [[float(v) for v in row] for row in c.F_xy]
        for a in range(2):
            for b in range(4):
                arr[i].F_xy[a][b] = F[a][b]
        arr[i].max_alt = float(c.max_alt)
        arr[i].width, arr[i].height = int(c.width), int(c.height)
        arr[i].sun_phi, arr[i].sun_theta = float(c.sun_phi), float(c.sun_theta)
        arr[i].shadow_w, arr[i].shadow_h = int(c.shadow_w), int(c.shadow_h)
        arr[i].shadow_scale = float(c.shadow_scale)
    return arr


def make_splats(means, scales, quats, opacity, rgb, n: int) -> ss_splats:
    """Splat descriptor of planar device tensors [C][n_pad] (fp32 or bf16)."""
    import torch
    dt = means.dtype
    assert all(t.dtype == dt for t in (scales, quats, opacity, rgb)), "one storage dtype"
    s = ss_splats()
    s.means, s.scales, s.quats, s.opacity, s.rgb = (ptr(means), ptr(scales), ptr(quats),
                                                    ptr(opacity), ptr(rgb))
    s.n = int(n)
    s.n_pad = int(means.shape[-1])
    s.dtype = SS_BF16 if dt == torch.bfloat16 else SS_F32
    return s


# ------------------------------------------------------------------------------ entry points
def workspace_size(splats, cams, n_cams, passes, opts, capacity) -> int:
    out = ctypes.c_size_t(0)
    _check(load().ss_workspace_size(ctypes.byref(splats), cams, n_cams, passes, ctypes.byref(opts),
                                    int(capacity), ctypes.byref(out)), "ss_workspace_size")
    return int(out.value)


def project_splats(splats, cams, n_cams, passes, dF, color, opts, ws, ws_bytes, capacity, stream=None):
    return _check(load().ss_project_splats(ctypes.byref(splats), cams, n_cams, passes, ptr(dF), ptr(color),
                                           ctypes.byref(opts), ptr(ws), int(ws_bytes), int(capacity),
                                           stream_ptr(stream)), "ss_project_splats")


def bin_and_sort(splats, cams, n_cams, passes, opts, ws, ws_bytes, capacity, sync_needed=True,
                 stream=None):
    """Returns (status, needed).  With sync_needed the stream is synchronised and the
    needed intersection count returned; SS_ERR_CAPACITY is returned, not raised."""
    needed = ctypes.c_int64(-1)
    st = load().ss_bin_and_sort(ctypes.byref(splats), cams, n_cams, passes, ctypes.byref(opts),
                                ptr(ws), int(ws_bytes), int(capacity),
                                ctypes.byref(needed) if sync_needed else None, stream_ptr(stream))
    _check(st, "ss_bin_and_sort", allow=(SS_ERR_CAPACITY,))
    return st, int(needed.value)


def rasterize_fwd(splats, cams, n_cams, passes, opts, io, ws, ws_bytes, capacity, stream=None):
    return _check(load().ss_rasterize_fwd(ctypes.byref(splats), cams, n_cams, passes,
                                          ctypes.byref(opts), io, ptr(ws), int(ws_bytes), int(capacity),
                                          stream_ptr(stream)), "ss_rasterize_fwd")


def rasterize_bwd(splats, cams, n_cams, passes, opts, io, grads, d_dF, d_color, ws, ws_bytes,
                  capacity, stream=None):
    """``grads`` None runs the per-pixel adjoint only (finish with project_bwd)."""
    g = None if grads is None else ctypes.byref(grads)
    return _check(load().ss_rasterize_bwd(ctypes.byref(splats), cams, n_cams, passes,
                                          ctypes.byref(opts), io, g, ptr(d_dF),
                                          ptr(d_color), ptr(ws), int(ws_bytes), int(capacity),
                                          stream_ptr(stream)), "ss_rasterize_bwd")


def project_bwd(splats, cams, n_cams, passes, opts, grads, d_dF, d_color, ws, ws_bytes, capacity, stream=None):
    return _check(load().ss_project_bwd(ctypes.byref(splats), cams, n_cams, passes, ctypes.byref(opts),
                                        ctypes.byref(grads), ptr(d_dF), ptr(d_color), ptr(ws), int(ws_bytes),
                                        int(capacity), stream_ptr(stream)), "ss_project_bwd")


def shadow_depth(splats, cams, n_cams, dF, opts, io, ws, ws_bytes, capacity, sync_needed=True, stream=None):
    needed = ctypes.c_int64(-1)
    st = load().ss_shadow_depth(ctypes.byref(splats), cams, n_cams, ptr(dF), ctypes.byref(opts), io,
                                ptr(ws), int(ws_bytes), int(capacity),
                                ctypes.byref(needed) if sync_needed else None, stream_ptr(stream))
    _check(st, "ss_shadow_depth", allow=(SS_ERR_CAPACITY,))
    return st, int(needed.value)


def frame_status(ws, ws_bytes, stream=None):
    """Returns (status, needed, nonfinite, walked, flags); synchronises the stream."""
    needed, nonfinite, walked, flags = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int32(0)
    st = load().ss_frame_status(ptr(ws), int(ws_bytes), ctypes.byref(needed), ctypes.byref(nonfinite),
                                ctypes.byref(walked), ctypes.byref(flags), stream_ptr(stream))
    return st, int(needed.value), int(nonfinite.value), int(walked.value), int(flags.value)


def render_fwd_noalloc(splats, cam, dF, color, opts, io, stream=None):
    """Allocation-free single-view forward (the library's static scratch).  Returns
    (status, needed); SS_ERR_CAPACITY is returned, not raised."""
    needed = ctypes.c_int64(-1)
    st = load().ss_render_fwd_noalloc(ctypes.byref(splats), cam, ptr(dF), ptr(color), ctypes.byref(opts), io,
                                      ctypes.byref(needed), stream_ptr(stream))
    _check(st, "ss_render_fwd_noalloc", allow=(SS_ERR_CAPACITY,))
    return st, int(needed.value)


def noalloc_scratch_bytes() -> int:
    return int(load().ss_noalloc_scratch_bytes())


def kernel_launches() -> int:
    return int(load().ss_kernel_launches())


def device_info():
    sms, arch = ctypes.c_int32(0), ctypes.c_int32(0)
    load().ss_device_info(ctypes.byref(sms), ctypes.byref(arch))
    return int(sms.value), int(arch.value)


# ------------------------------------------------------------------------------ shading (K7)
def default_shade_opts(**overrides) -> ss_shade_opts:
    o = ss_shade_opts()
    load().ss_default_shade_opts(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def shade_io_array(views: Sequence[dict]) -> ctypes.Array:
    """ss_shade_io per view from dicts of tensors (keys as the struct's fields; missing = NULL)."""
    arr = (ss_shade_io * len(views))()
    for i, v in enumerate(views):
        for name, _ in ss_shade_io._fields_:
            setattr(arr[i], name, ptr(v.get(name)))
    return arr


def shade_fwd(cams, n_cams: int, dF, La, opts: ss_shade_opts, io, stream=None) -> None:
    _check(load().ss_shade_fwd(cams, n_cams, ptr(dF), ptr(La), ctypes.byref(opts), io, stream_ptr(stream)),
           "ss_shade_fwd")


def shade_bwd(cams, n_cams: int, dF, La, opts: ss_shade_opts, io, d_La=None, d_dF=None, stream=None) -> None:
    _check(load().ss_shade_bwd(cams, n_cams, ptr(dF), ptr(La), ctypes.byref(opts), io, ptr(d_La), ptr(d_dF),
                               stream_ptr(stream)), "ss_shade_bwd")


# ------------------------------------------------------------------------------ depth normal (K8)
def dnormal_io_array(views: Sequence[dict]) -> ctypes.Array:
    arr = (ss_dnormal_io * len(views))()
    for i, v in enumerate(views):
        for name, _ in ss_dnormal_io._fields_:
            setattr(arr[i], name, ptr(v.get(name)))
    return arr


def depth_normal_fwd(cams, n_cams: int, dF, alpha_eps: float, io, stream=None) -> None:
    _check(load().ss_depth_normal_fwd(cams, n_cams, ptr(dF), float(alpha_eps), io, stream_ptr(stream)),
           "ss_depth_normal_fwd")


def depth_normal_bwd(cams, n_cams: int, dF, alpha_eps: float, io, d_dF=None, stream=None) -> None:
    _check(load().ss_depth_normal_bwd(cams, n_cams, ptr(dF), float(alpha_eps), io, ptr(d_dF), stream_ptr(stream)),
           "ss_depth_normal_bwd")


# ------------------------------------------------------------------------------ optimiser step
def default_adam_opts(**overrides) -> ss_adam_opts:
    o = ss_adam_opts()
    load().ss_default_adam_opts(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def default_mcmc_opts(**overrides) -> ss_mcmc_opts:
    o = ss_mcmc_opts()
    load().ss_default_mcmc_opts(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def make_params(means, log_scales, quats, logit_opacity, rgb) -> ss_splat_params:
    """ss_splat_params over planar fp32 [C, n_pad] tensors (raw parameters or Adam moments)."""
    import torch

    ts = (means, log_scales, quats, logit_opacity, rgb)
    for t in ts:
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError("parameter rows must be contiguous float32 [C, n_pad] tensors")
    p = ss_splat_params()
    p.means, p.log_scales, p.quats, p.logit_opacity, p.rgb = (ptr(t) for t in ts)
    p.n_pad = int(means.shape[-1])
    return p


def adam_step(params: ss_splat_params, exp_avg: ss_splat_params, exp_avg_sq: ss_splat_params, grads,
              storage, opts: ss_adam_opts, stream=None) -> None:
    _check(load().ss_adam_step(ctypes.byref(params), ctypes.byref(exp_avg), ctypes.byref(exp_avg_sq),
                               ctypes.byref(grads), ctypes.byref(storage), ctypes.byref(opts), stream_ptr(stream)),
           "ss_adam_step")


def adam_flat(param, exp_avg, exp_avg_sq, grad, lr: float, opts: ss_adam_opts, stream=None) -> None:
    _check(load().ss_adam_flat(ptr(param), ptr(exp_avg), ptr(exp_avg_sq), ptr(grad), int(param.numel()), float(lr),
                               ctypes.byref(opts), stream_ptr(stream)), "ss_adam_flat")


def mcmc_workspace_size(cap: int) -> int:
    b = ctypes.c_size_t(0)
    _check(load().ss_mcmc_workspace_size(int(cap), ctypes.byref(b)), "ss_mcmc_workspace_size")
    return int(b.value)


def mcmc_relocate(params: ss_splat_params, exp_avg: ss_splat_params, exp_avg_sq: ss_splat_params, storage,
                  cap: int, opts: ss_mcmc_opts, ws, d_stats=None, stream=None) -> int:
    """Relocation and growth in place; returns the new active count (synchronises the stream)."""
    n_after = ctypes.c_int64(0)
    _check(load().ss_mcmc_relocate(ctypes.byref(params), ctypes.byref(exp_avg), ctypes.byref(exp_avg_sq),
                                   ctypes.byref(storage), int(cap), ctypes.byref(opts), ptr(ws), int(ws.numel()),
                                   ctypes.byref(n_after), ptr(d_stats), stream_ptr(stream)), "ss_mcmc_relocate")
    return int(n_after.value)


# ------------------------------------------------------------------------------ initialisation
def default_init_opts(**overrides) -> ss_init_opts:
    o = ss_init_opts()
    load().ss_default_init_opts(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def make_dsm(heights, rgb, x0: float, y0: float, gsd: float) -> ss_dsm:
    """ss_dsm over a device heights tensor (H, W) fp32 and an optional rgb (3, H, W) fp32."""
    d = ss_dsm()
    d.heights, d.rgb = ptr(heights), ptr(rgb)
    d.height_px, d.width = int(heights.shape[0]), int(heights.shape[1])
    d.x0, d.y0, d.gsd = float(x0), float(y0), float(gsd)
    return d


def init_workspace_size(dsm: ss_dsm, n: int) -> int:
    b = ctypes.c_size_t(0)
    _check(load().ss_init_workspace_size(ctypes.byref(dsm), int(n), ctypes.byref(b)), "ss_init_workspace_size")
    return int(b.value)


def dsm_init(dsm: ss_dsm, opts: ss_init_opts, out, ws, stream=None) -> None:
    _check(load().ss_dsm_init(ctypes.byref(dsm), ctypes.byref(opts), ctypes.byref(out), ptr(ws), int(ws.numel()),
                              stream_ptr(stream)), "ss_dsm_init")
