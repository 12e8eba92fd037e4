#!/usr/bin/env python
"""Benchmark of the GB300 affine 2DGS rasterizer (forward + backward, Mpix/s).

Default workload ("batched"): 1M splats over 1 km^2, 16 views of uneven size
(1024^2 - 2048^2) with camera deltas, plus the sun-view shadow-depth pass of
every view at half resolution; splat attributes stored in BF16; one step =
projection, binning, forward and backward of all 32 targets, replayed from two
CUDA graphs (forward part, backward part) with persistent launches.  Mpix/s counts main-view pixels per
forward+backward step.  Beside it: the same scene as 16 plain FP32 single-view
calls, an end-to-end run through the public API with host buffers, live
per-kernel timing for the roofline, and the FP64 oracle on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank renders its own replica of the workload (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Mpix/s at 1M splats (batched BF16 vs plain FP32), % of roofline"
UNIT = "Mpix/s"
# FP32 operations per contributing (pixel, splat) pair, counted from the kernel source
# (FADD/FMUL = 1, FFMA = 2; the exp and the reciprocal are MUFU ops, not counted):
#   forward: pair evaluation 20 + compositing 21
#   backward: pair evaluation 20 + adjoint 63 + accumulation of 16 gradient fields 16
FLOPS_FWD_PER_PAIR = 41
FLOPS_BWD_PER_PAIR = 99
# with the distortion of the blending weights: forward + 6 (its running sum), backward + 18 (its
# partials in the weight and the depth and the running weighted depth behind the splat)
FLOPS_FWD_PER_PAIR_DIST = 47
FLOPS_BWD_PER_PAIR_DIST = 117
FP32_LANES_PER_SM = 128

WORKLOAD_TEXT = {
    "batched": "1M splats over 1 km^2; 16 views of uneven size 1024^2-2048^2 with camera deltas; "
               "a sun-view shadow-depth pass per view at half resolution",
    "single": "500k splats over 1 km^2; one 2048^2 view with colour correction plus a 1024^2 sun view",
    "small": "4096 splats over 100 m; one 128^2 view plus a 64^2 sun view",
    "full": "4M splats over 2x2 km; 32 views at 2048^2 with deltas and colour correction, each with a "
            "1024^2 sun view",
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched", choices=list(WORKLOAD_TEXT))
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 single-view arm")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (16x16, batch 256)")
    ap.add_argument("--no-distortion", action="store_true",
                    help="skip timing the step with the distortion plane")
    ap.add_argument("--storage", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--profile", action="store_true",
                    help="short run for a profiler: no tuning, plain, e2e, CPU or distortion arms")
    return ap.parse_args()


# ------------------------------------------------------------------------------ distributed
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        import torch.distributed as dist
        if self.world > 1 and not dist.is_initialized():
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


def gpu_smi_id(torch, dev):
    try:
        p = torch.cuda.get_device_properties(dev)
        bus = getattr(p, "pci_bus_id", None)
        dom = getattr(p, "pci_domain_id", 0)
        did = getattr(p, "pci_device_id", 0)
        if bus is not None:
            return f"{dom:08X}:{bus:02X}:{did:02X}.0"
    except Exception:
        pass
    return None


# ------------------------------------------------------------------------------ helpers
def upload_splats(torch, scene, dtype):
    from paper_2606_28581_gb300.frame import n_pad_of, pad_planar
    n_pad = n_pad_of(scene.n)
    t = lambda a: pad_planar(torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().to(dtype), n_pad)
    return dict(means=t(scene.means), scales=t(scene.scales), quats=t(scene.quats),
                opacity=t(scene.opacity[None]), rgb=t(scene.rgb))


def make_upstream(torch, targets, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    ups = []
    for t in targets:
        r = lambda *s: torch.randn(*s, device="cuda", generator=g)
        if t.sun:
            ups.append(dict(depth=r(t.height, t.width), alpha=r(t.height, t.width)))
        else:
            ups.append(dict(rgb=r(3, t.height, t.width), depth=r(t.height, t.width),
                            normal=r(3, t.height, t.width), alpha=r(t.height, t.width)))
    return ups


def time_loop(torch, fn, steps):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(steps):
        fn()
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / steps


def profiles_traffic(kernel: str):
    """Per-launch DRAM traffic of `kernel` from the committed ncu summary, if the summary was
    taken on the current kernel sources (fingerprint of the listed files, concatenated); else
    None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for ln in open(path):
        if ":" in ln:
            k, v = ln.split(":", 1)
            vals[k.strip()] = v.strip()
    h = hashlib.sha256()
    for name in vals.get("source", "raster_impl.cuh").split():
        src = os.path.join(ROOT, "paper_2606_28581_gb300", "csrc", name)
        if not os.path.exists(src):
            return None
        h.update(open(src, "rb").read())
    if vals.get("source_sha256_16") != h.hexdigest()[:16]:
        return None
    try:
        return float(vals["bytes_per_launch_full"])
    except (KeyError, ValueError):
        return None


def hbm_peak_gbs():
    """Measured copy bandwidth of this machine's GPUs (MEASURED_PEAKS.json), else the fallback."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def loaded_clock_mhz():
    """The median SM clock the machine's GPUs held under a seconds-long dense load
    (MEASURED_PEAKS.json), else the fallback of 1485 MHz."""
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(peaks["clocks_under_load"]["sm_mhz_median"])
    except Exception:
        return 1485.0


def measure_shade(torch, step, reps: int):
    """Forward and backward of the shading (K7) over every main view of the step, on the step's
    rasterized planes, with CUDA events; HBM roofline from the algorithmic bytes per main pixel
    (forward: rgb, depth, alpha read, image written = 32 B; backward: d_image, rgb, depth, alpha
    read, d_rgb read and written = 56 B) plus 8 B per sun pixel.  Data-dependent traffic (the
    shadowed pixels' depth and alpha gradients, the sun-view atomics) is not counted."""
    from paper_2606_28581_gb300 import _lib as L
    f, out = step.frame, step.out
    V = f.n_cams
    if len(f.targets) != 2 * V:
        return None
    dev = out.rgb[0].device
    La = torch.full((V, 3), 0.3, device=dev)
    views_f, views_b = [], []
    main_px = sun_px = 0
    for c in range(V):
        base = dict(rgb=out.rgb[c], depth=out.depth[c], alpha=out.alpha[c], sun_depth=out.depth[V + c],
                    sun_alpha=out.alpha[V + c])
        main_px += out.depth[c].numel()
        sun_px += out.depth[V + c].numel()
        views_f.append(dict(base, image=torch.empty_like(out.rgb[c])))
        views_b.append(dict(base, d_image=torch.randn_like(out.rgb[c]), d_rgb=torch.zeros_like(out.rgb[c]),
                            d_depth=torch.zeros_like(out.depth[c]), d_alpha=torch.zeros_like(out.alpha[c]),
                            d_sun_depth=torch.zeros_like(out.depth[V + c]),
                            d_sun_alpha=torch.zeros_like(out.alpha[V + c])))
    io_f, io_b = L.shade_io_array(views_f), L.shade_io_array(views_b)
    opts = L.default_shade_opts()
    d_La = torch.zeros(V, 3, device=dev)
    d_dF = torch.zeros(V, 2, 4, device=dev)
    dF = step.dF
    fwd = lambda: L.shade_fwd(f.cams, V, dF, La, opts, io_f)
    bwd = lambda: L.shade_bwd(f.cams, V, dF, La, opts, io_b, d_La, d_dF)
    fwd(); bwd()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    acc = np.zeros(2)
    for _ in range(reps):
        ev[0].record(); fwd(); ev[1].record(); bwd(); ev[2].record()
        torch.cuda.synchronize()
        acc += [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])]
    fms, bms = acc / reps
    peak, basis = hbm_peak_gbs()
    bf, bb = main_px * 32 + sun_px * 8, main_px * 56 + sun_px * 8
    return {"bound": "hbm", "fwd_ms": float(fms), "bwd_ms": float(bms), "bytes_fwd": int(bf), "bytes_bwd": int(bb),
            "fwd_gbs": bf / (fms * 1e-3) / 1e9, "bwd_gbs": bb / (bms * 1e-3) / 1e9, "peak_gbs": peak,
            "peak_basis": basis, "fwd_frac": bf / (fms * 1e-3) / 1e9 / peak,
            "bwd_frac": bb / (bms * 1e-3) / 1e9 / peak}


def measure_distortion(torch, mk, ups, reps: int, walked: int, base_ms: dict, peak_tflops: float):
    """The same batched step with the distortion plane written by the forward and an upstream
    distortion gradient in the backward: the step through its graphs, and the forward and
    backward kernels with CUDA events, against the step without it."""
    targets_ups = []
    g = torch.Generator(device="cuda")
    g.manual_seed(4321)
    for u in ups:
        u = dict(u)
        if "rgb" in u:  # a main target
            u["distort"] = torch.randn(*u["depth"].shape, device="cuda", generator=g)
        targets_ups.append(u)
    step = mk(targets_ups)
    step.capture()
    for _ in range(3):
        step.replay()
    ms = time_loop(torch, step.replay, reps)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    acc = np.zeros(2)
    for _ in range(reps):
        step.forward_part()
        step.zero_grads()
        ev[0].record(); step.forward(); ev[1].record(); step.backward_pixels(); ev[2].record()
        torch.cuda.synchronize()
        acc += [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])]
    fms, bms = acc / reps
    st = step.check()[0]
    del step
    torch.cuda.empty_cache()
    if st != 0:
        raise RuntimeError(f"distortion step status {st}")
    bw = walked * FLOPS_BWD_PER_PAIR_DIST / (bms * 1e-3) / 1e12
    return {"step_ms": float(ms), "rasterize_fwd_ms": float(fms), "rasterize_bwd_ms": float(bms),
            "step_over_plain_step": float(ms / base_ms["step"]),
            "fwd_over_plain_fwd": float(fms / base_ms["rasterize_fwd"]),
            "bwd_over_plain_bwd": float(bms / base_ms["rasterize_bwd"]),
            "bwd_roofline": {"bound": "alu", "achieved": bw, "peak": peak_tflops, "unit": "TFLOP/s",
                             "frac": bw / peak_tflops, "flops_per_pair": FLOPS_BWD_PER_PAIR_DIST}}


def measure_optimizer(torch, n: int, grads: dict, storage_dtype, reps: int):
    """The fused Adam step (with the position noise) over the step's n splats, with CUDA events,
    and one 3DGS-MCMC relocation with 5 % growth and about 5 % dead splats (host timer: the call
    synchronises).  HBM roofline of the Adam step from its algorithmic bytes per splat: 13
    gradients, 13 raw values and 26 moments read, 13 raw values and 26 moments written (4 B
    each), and 13 stored values written (2 B in BF16, 4 B in FP32)."""
    from paper_2606_28581_gb300 import _lib as L
    from paper_2606_28581_gb300.frame import n_pad_of
    cap = n + n // 20
    n_pad = max(n_pad_of(cap), int(grads["means"].shape[-1]))
    g = torch.Generator(device="cuda")
    g.manual_seed(99)
    rows = dict(means=3, log_scales=2, quats=4, logit_opacity=1, rgb=3)
    mk = lambda s: {k: torch.randn(c, n_pad, device="cuda", generator=g) * s for k, c in rows.items()}
    raw, m, v = mk(0.3), mk(1e-2), mk(1e-2)
    v = {k: t.abs() for k, t in v.items()}
    raw["log_scales"].mul_(0.1).add_(-6.0)
    gpad = {k: torch.zeros(t.shape[0], n_pad, device="cuda") for k, t in grads.items()}
    for k, t in grads.items():
        gpad[k][:, : t.shape[-1]] = t
    st = {k: torch.zeros(c, n_pad, device="cuda", dtype=storage_dtype)
          for k, c in dict(means=3, scales=2, quats=4, opacity=1, rgb=3).items()}
    storage = L.make_splats(st["means"], st["scales"], st["quats"], st["opacity"], st["rgb"], n)
    P = lambda d: L.make_params(d["means"], d["log_scales"], d["quats"], d["logit_opacity"], d["rgb"])
    pp, pm, pv = P(raw), P(m), P(v)
    gs = L.ss_splat_grads()
    gs.means, gs.scales, gs.quats, gs.opacity, gs.rgb = (L.ptr(gpad[k]) for k in ("means", "scales", "quats",
                                                                                   "opacity", "rgb"))
    gs.n_pad = n_pad
    it = [0]

    def adam():
        it[0] += 1
        L.adam_step(pp, pm, pv, gs, storage, L.default_adam_opts(step=it[0]))

    for _ in range(3):
        adam()
    ms = time_loop(torch, adam, reps)
    per_splat = 4 * (13 + 13 + 26 + 13 + 26) + 13 * (2 if storage_dtype == torch.bfloat16 else 4)
    peak, basis = hbm_peak_gbs()
    gbs = n * per_splat / (ms * 1e-3) / 1e9
    # relocation: about 5 % of the splats dead, 5 % growth
    ws = torch.empty(L.mcmc_workspace_size(cap), dtype=torch.uint8, device="cuda")
    logit0 = raw["logit_opacity"].clone()
    dead = torch.rand(n_pad, device="cuda", generator=g) < 0.05
    rl = []
    for r in range(3):
        raw["logit_opacity"].copy_(logit0)
        raw["logit_opacity"][0, dead] = -8.0
        st["opacity"].copy_(torch.sigmoid(raw["logit_opacity"]).to(storage_dtype))
        storage.n = n
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_after = L.mcmc_relocate(pp, pm, pv, storage, cap, L.default_mcmc_opts(step=r), ws)
        torch.cuda.synchronize()  # the call returns before its last kernels finish
        rl.append((time.perf_counter() - t0) * 1e3)
    return {"bound": "hbm", "splats": n, "adam_ms": float(ms), "adam_bytes_per_splat": per_splat,
            "adam_gbs": gbs, "peak_gbs": peak, "peak_basis": basis, "adam_frac": gbs / peak,
            "relocate_ms": float(np.median(rl)), "relocate_n_after": int(n_after), "relocate_cap": int(cap),
            "relocate_note": "host-timed from the call to the end of its last kernel (a synchronisation after it)"}


def measure_init(torch, reps: int):
    """The geometry-aware initialisation over a 2048 x 2048 DSM of 1 km^2 (0.5 m) with 1M
    samples, with CUDA events around the whole call (weights, scan, draws, cell sort, kNN)."""
    import scenegen
    from paper_2606_28581_gb300 import _lib as L
    from paper_2606_28581_gb300.frame import n_pad_of
    dsm = scenegen.make_dsm(size_px=2048, extent_m=1000.0, seed=6)
    Z = torch.from_numpy(dsm.height).cuda()
    rgb = torch.from_numpy(dsm.rgb).cuda()
    d = L.make_dsm(Z, rgb, dsm.x0, dsm.y0, dsm.gsd)
    n = 1_000_000
    n_pad = n_pad_of(n)
    st = {k: torch.zeros(c, n_pad, device="cuda", dtype=torch.bfloat16)
          for k, c in dict(means=3, scales=2, quats=4, opacity=1, rgb=3).items()}
    out = L.make_splats(st["means"], st["scales"], st["quats"], st["opacity"], st["rgb"], n)
    ws = torch.empty(L.init_workspace_size(d, n), dtype=torch.uint8, device="cuda")
    opts = L.default_init_opts()
    run = lambda: L.dsm_init(d, opts, out, ws)
    run()
    ms = time_loop(torch, run, reps)
    return {"dsm_px": [2048, 2048], "samples": n, "ms": float(ms), "msamples_per_s": n / (ms * 1e-3) / 1e6,
            "storage": "bf16"}


def measure_depth_normal(torch, step, reps: int):
    """Forward and backward of the depth-gradient normal (K8) over every main view of the step;
    HBM roofline from the algorithmic bytes per main pixel (forward: depth and alpha read, N
    written = 20 B; backward: dN, depth, alpha read and the depth and alpha gradients read and
    written = 36 B; the neighbours' reads and the atomics' re-reads hit L1/L2)."""
    from paper_2606_28581_gb300 import _lib as L
    f, out = step.frame, step.out
    V = f.n_cams
    main = [i for i, t in enumerate(f.targets) if not t.sun]
    if len(main) != V:
        return None
    views_f, views_b = [], []
    px = 0
    for c in main:
        d, a = out.depth[c], out.alpha[c]
        px += d.numel()
        views_f.append(dict(depth=d, alpha=a, normal=torch.empty(3, *d.shape, device=d.device)))
        views_b.append(dict(depth=d, alpha=a, d_normal=torch.randn(3, *d.shape, device=d.device),
                            d_depth=torch.zeros_like(d), d_alpha=torch.zeros_like(a)))
    io_f, io_b = L.dnormal_io_array(views_f), L.dnormal_io_array(views_b)
    d_dF = torch.zeros(V, 2, 4, device=out.depth[0].device)
    fwd = lambda: L.depth_normal_fwd(f.cams, V, step.dF, 1e-3, io_f)
    bwd = lambda: L.depth_normal_bwd(f.cams, V, step.dF, 1e-3, io_b, d_dF)
    fwd(); bwd()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    acc = np.zeros(2)
    for _ in range(reps):
        ev[0].record(); fwd(); ev[1].record(); bwd(); ev[2].record()
        torch.cuda.synchronize()
        acc += [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])]
    fms, bms = acc / reps
    peak, basis = hbm_peak_gbs()
    bf, bb = px * 20, px * 36
    return {"bound": "hbm", "fwd_ms": float(fms), "bwd_ms": float(bms), "bytes_fwd": int(bf), "bytes_bwd": int(bb),
            "fwd_gbs": bf / (fms * 1e-3) / 1e9, "bwd_gbs": bb / (bms * 1e-3) / 1e9, "peak_gbs": peak,
            "peak_basis": basis, "fwd_frac": bf / (fms * 1e-3) / 1e9 / peak,
            "bwd_frac": bb / (bms * 1e-3) / 1e9 / peak}


def measure_config(torch, name: str, storage_dtype, steps: int, warmup: int = 3):
    """Another configuration of the same path, timed alone: the workload's main views and sun
    views as one BatchedStep (two CUDA graphs, persistent launches, 16 x 16 tiles), forward and
    backward, with CUDA events.  Mpix/s counts main-view pixels per forward+backward step."""
    import scenegen
    from paper_2606_28581_gb300 import _lib as L
    from paper_2606_28581_gb300.batched import BatchedStep
    from paper_2606_28581_gb300.frame import Frame
    scene = scenegen.workload(name, seed=0)
    cams = scene.cameras
    passes = L.SS_PASS_MAIN | L.SS_PASS_SUN
    splats = upload_splats(torch, scene, storage_dtype)
    dF = torch.from_numpy(np.stack([c.dF_xy for c in cams]).astype(np.float32)).cuda()
    color = torch.from_numpy(np.stack([c.color for c in cams]).astype(np.float32)).cuda()
    ups = make_upstream(torch, Frame(cams, passes).targets, 4321)
    step = BatchedStep(cams, splats, scene.n, dF, color, ups, passes=passes, opts=L.default_opts(persistent=1))
    step.capture()
    for _ in range(warmup):
        step.replay()
    ms = time_loop(torch, step.replay, steps)
    st = step.check()[0]
    if st != L.SS_OK:
        raise RuntimeError(f"{name} step status {L.status_string(st)}")
    main_px, sun_px = step.main_pixels, step.sun_pixels
    out = {"workload": WORKLOAD_TEXT[name], "n_splats": scene.n,
           "storage": "bf16" if storage_dtype == torch.bfloat16 else "fp32", "value": main_px / (ms * 1e-3) / 1e6,
           "unit": UNIT, "ms_per_step": ms, "steps": steps, "main_pixels": main_px, "sun_pixels": sun_px}
    del step
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------------------ oracle arm
def oracle_sample(scene, seconds_target: float, seed: int = 0, parts: bool = False):
    """Time the FP64 oracle (forward + backward) on crops of view 0, growing the crop until
    one sample takes about `seconds_target`.  Returns (Mpix/s, crop, seconds, threads), and with
    `parts` also the forward's own Mpix/s."""
    import oracle
    s64 = oracle.SceneF64.of(scene)
    cam = scene.cameras[0]
    rng = np.random.default_rng(seed)
    side = 64
    while True:
        w = min(side, cam.width)
        h = min(side, cam.height)
        x0 = (cam.width - w) // 2
        y0 = (cam.height - h) // 2
        g = dict(rgb=rng.normal(size=(3, h, w)), depth=rng.normal(size=(h, w)),
                 normal=rng.normal(size=(3, h, w)), alpha=rng.normal(size=(h, w)))
        t0 = time.perf_counter()
        oracle.render(s64, cam, crop=(x0, y0, w, h), color=cam.color)
        t1 = time.perf_counter()
        oracle.backward(s64, cam, g, crop=(x0, y0, w, h), color=cam.color)
        dt = time.perf_counter() - t0
        if dt >= seconds_target or (w == cam.width and h == cam.height) or side >= 4096:
            r = ((w * h) / dt / 1e6, (x0, y0, w, h), dt, oracle.num_threads())
            return r + ((w * h) / (t1 - t0) / 1e6,) if parts else r
        side = int(side * min(4.0, max(1.3, math.sqrt(seconds_target / max(dt, 1e-3)))))


def run_reference(args, dist):
    """The oracle as the reference arm: each step is forward + backward of the FP64 oracle
    on a bounded crop of the same workload, on the host cores."""
    import scenegen
    if dist.rank != 0:
        return 0
    scene = scenegen.workload(args.workload, seed=0)
    main_px = sum(c.width * c.height for c in scene.cameras)
    # size one step to about 1.5 s so that warm-up + steps end within a few minutes
    per_step = max(0.5, min(3.0, 150.0 / max(1, args.steps + args.warmup)))
    _, crop, _, threads = oracle_sample(scene, per_step)
    import oracle
    s64 = oracle.SceneF64.of(scene)
    cam = scene.cameras[0]
    x0, y0, w, h = crop
    rng = np.random.default_rng(1)
    g = dict(rgb=rng.normal(size=(3, h, w)), depth=rng.normal(size=(h, w)),
             normal=rng.normal(size=(3, h, w)), alpha=rng.normal(size=(h, w)))

    def step():
        oracle.render(s64, cam, crop=crop, color=cam.color)
        oracle.backward(s64, cam, g, crop=crop, color=cam.color)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    value = (w * h) / dt / 1e6
    sample = f"{w}x{h} px crop of view 0 of the '{args.workload}' workload per step, all {scene.n} splats"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload], "n_splats": scene.n, "main_pixels": main_px},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ our arm
def run_ours(args, dist):
    import torch
    import scenegen
    from paper_2606_28581_gb300 import _lib as L
    from paper_2606_28581_gb300.batched import BatchedStep, autotune, workload_key
    from paper_2606_28581_gb300.frame import Frame, Outputs, grads_struct, zero_grads

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    dev = dist.local
    torch.cuda.set_device(dev)
    dist.init("nccl")
    L.load()
    sms, arch = L.device_info()
    if args.profile:
        args.no_plain = args.no_cpu = args.no_e2e = args.no_tune = args.no_distortion = True

    scene = scenegen.workload(args.workload, seed=dist.rank)
    cams = scene.cameras
    passes = L.SS_PASS_MAIN | L.SS_PASS_SUN
    storage = torch.bfloat16 if args.storage == "bf16" else torch.float32
    splats = upload_splats(torch, scene, storage)
    dF = torch.from_numpy(np.stack([c.dF_xy for c in cams]).astype(np.float32)).cuda()
    color = torch.from_numpy(np.stack([c.color for c in cams]).astype(np.float32)).cuda()
    probe = Frame(cams, passes)
    ups = make_upstream(torch, probe.targets, 1234 + dist.rank)
    main_px = sum(t.width * t.height for t in probe.targets if not t.sun)
    sun_px = sum(t.width * t.height for t in probe.targets if t.sun)

    # ---- autotuned options (tile shape, batch), persistent launches
    mk = lambda o: BatchedStep(cams, splats, scene.n, dF, color, ups, passes=passes, opts=o)
    tune = None
    if args.no_tune:
        opts = L.default_opts(persistent=1)
    else:
        opts, tune = autotune(mk, workload_key(cams, scene.n, args.storage, passes), log=log)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    step = mk(opts)
    n_before = L.kernel_launches()
    step.capture()
    launches_per_step = L.kernel_launches() - n_before
    # capture ran one eager warm-up step plus the captured one
    launches_per_step = launches_per_step // 2

    for _ in range(args.warmup):
        step.replay()
    torch.cuda.synchronize()
    st, needed, walked, flags = step.check()
    if st != L.SS_OK:
        raise RuntimeError(f"frame status {L.status_string(st)} (needed {needed}, flags {flags})")

    clk = ClockSampler(gpu_smi_id(torch, dev))
    dist.barrier()
    clk.start()
    ms = time_loop(torch, step.replay, args.steps)
    clocks = clk.stop()
    # device memory of the timed step: inputs, outputs, upstream planes, gradients, workspace
    peak_hbm_gb = torch.cuda.max_memory_allocated() / 1e9
    dist.barrier()
    ms_max = dist.max(ms)
    total_px = dist.sum(main_px)
    value = total_px / (ms_max * 1e-3) / 1e6
    st, needed, _, flags = step.check()
    if st != L.SS_OK:
        raise RuntimeError(f"frame status after timing: {L.status_string(st)}")
    # the algorithmic work (walked pairs) from a counting forward outside the timed region
    walked = step.count_walked()

    # ---- live per-kernel timing (same kernels and launch configuration, eager, events between)
    k_steps = max(3, min(args.steps, 20))
    names = ["project", "bin_and_sort", "rasterize_fwd", "rasterize_bwd", "project_bwd"]
    phases = [step.project, step.bin, step.forward, step.backward_pixels, step.backward_project]
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(phases) + 1)]
    acc = np.zeros(len(phases))
    for _ in range(k_steps):
        step.zero_grads()
        evs[0].record()
        for i, f in enumerate(phases):
            f()
            evs[i + 1].record()
        torch.cuda.synchronize()
        acc += [evs[i].elapsed_time(evs[i + 1]) for i in range(len(phases))]
    phase_ms = {n: float(a / k_steps) for n, a in zip(names, acc)}
    loaded_mhz = loaded_clock_mhz()
    clock_mhz = clocks["sm_mhz"] if clocks else loaded_mhz
    peak_tflops = sms * FP32_LANES_PER_SM * 2 * clock_mhz * 1e6 / 1e12
    flops = {"rasterize_fwd": walked * FLOPS_FWD_PER_PAIR, "rasterize_bwd": walked * FLOPS_BWD_PER_PAIR}
    dom = max(("rasterize_fwd", "rasterize_bwd"), key=lambda k: phase_ms[k])
    achieved = flops[dom] / (phase_ms[dom] * 1e-3) / 1e12
    # the committed per-launch traffic is scaled to the 16-view batched step
    traffic = profiles_traffic("raster_bwd") if dom == "rasterize_bwd" and args.workload == "batched" else None
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": traffic,
                "flops_per_launch": flops[dom], "walked_pairs": walked,
                "flops_per_pair": FLOPS_BWD_PER_PAIR if dom == "rasterize_bwd" else FLOPS_FWD_PER_PAIR,
                "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {clock_mhz:.0f} MHz "
                              f"(median SM clock sampled during the timed region)",
                "frac_at_max_clock": achieved / (sms * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12),
                "loaded_clock_mhz": loaded_mhz,
                "frac_at_loaded_clock": achieved / (sms * FP32_LANES_PER_SM * 2 * loaded_mhz * 1e6 / 1e12),
                "phase_ms": phase_ms}

    # ---- sun visibility and image formation (K7), depth-gradient normals (K8), timed alone
    shade = measure_shade(torch, step, k_steps)
    dnormal = measure_depth_normal(torch, step, k_steps)
    optimizer = measure_optimizer(torch, scene.n, step.grads, storage, k_steps)
    init = measure_init(torch, 3)
    # the other configurations of the path: the single 2048^2 view with its shadow pass in FP32
    # and in BF16 storage, and the small 128^2 view (parity of each against the oracle is checked
    # by the test suite, not here)
    single = small = None
    if args.workload == "batched" and not args.profile:
        s32 = measure_config(torch, "single", torch.float32, 20)
        s16 = measure_config(torch, "single", torch.bfloat16, 20)
        single = {"fp32": s32, "bf16": s16, "bf16_over_fp32": s16["value"] / s32["value"]}
        small = measure_config(torch, "small", torch.float32, 50)
    distortion = None
    if not args.no_distortion:
        mk_d = lambda u: BatchedStep(cams, splats, scene.n, dF, color, u, passes=passes, opts=opts,
                                     distortion=True)
        distortion = measure_distortion(torch, mk_d, ups, k_steps, walked, dict(phase_ms, step=ms), peak_tflops)

    # ---- plain FP32 single-view arm: the same scene as one plain call sequence per view
    plain = None
    if not args.no_plain:
        splats32 = upload_splats(torch, scene, torch.float32)
        s32 = L.make_splats(splats32["means"], splats32["scales"], splats32["quats"], splats32["opacity"],
                            splats32["rgb"], scene.n)
        frames, outs, ios = [], [], []
        for v, c in enumerate(cams):
            f = Frame([c], passes, L.default_opts())
            f.project_and_bin(s32, dF[v:v + 1].contiguous(), color[v:v + 1].contiguous(), sync=True)
            f.ensure_workspace(s32, int(f.needed * 1.1) + 4096)
            o = Outputs(f.targets, f.device)
            u = [ups[v], ups[len(cams) + v]]
            frames.append(f)
            outs.append(o)
            ios.append((o.io_array(), o.io_array(u)))
        g32 = zero_grads(splats32["means"].shape[-1], "cuda")
        gs = grads_struct(g32)
        dFv = [dF[v:v + 1].contiguous() for v in range(len(cams))]
        colv = [color[v:v + 1].contiguous() for v in range(len(cams))]
        ddF = torch.zeros(len(cams), 2, 4, device="cuda")
        dcol = torch.zeros(len(cams), 3, 4, device="cuda")

        def plain_step():
            for g in g32.values():
                g.zero_()
            for v, f in enumerate(frames):
                L.project_splats(s32, f.cams, 1, passes, dFv[v], colv[v], f.opts, f.ws, f.ws_bytes, f.capacity)
                L.bin_and_sort(s32, f.cams, 1, passes, f.opts, f.ws, f.ws_bytes, f.capacity, sync_needed=False)
                L.rasterize_fwd(s32, f.cams, 1, passes, f.opts, ios[v][0], f.ws, f.ws_bytes, f.capacity)
                L.rasterize_bwd(s32, f.cams, 1, passes, f.opts, ios[v][1], gs, ddF[v:v + 1],
                                dcol[v:v + 1], f.ws, f.ws_bytes, f.capacity)

        for _ in range(max(1, min(args.warmup, 3))):
            plain_step()
        p_steps = max(3, min(args.steps, 20))
        pms = time_loop(torch, plain_step, p_steps)
        for f in frames:
            stf = f.status()[0]
            if stf != L.SS_OK:
                raise RuntimeError(f"plain frame status {L.status_string(stf)}")
        plain = {"value": main_px / (pms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": pms, "steps": p_steps,
                 "storage": "fp32", "launch": f"{len(frames)} sequential single-view call sequences (eager, one "
                                               "warp per half tile, 16x16 tiles)"}
        del frames, outs, ios, splats32
        torch.cuda.empty_cache()

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda t: t.detach().cpu().pin_memory()
        h_in = {k: pin(v) for k, v in splats.items()}
        h_in["dF"], h_in["color"] = pin(dF), pin(color)
        h_ups = [{k: pin(v) for k, v in u.items()} for u in ups]
        h_out = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in step.grads.items()}
        h_out["d_dF"] = torch.empty_like(step.d_dF, device="cpu").pin_memory()
        h_out["d_color"] = torch.empty_like(step.d_color, device="cpu").pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in h_in.values())
        h2d += sum(t.numel() * t.element_size() for u in h_ups for t in u.values())
        d2h = sum(t.numel() * t.element_size() for t in h_out.values())

        def e2e_step():
            # the public host-buffer step: upstream planes arrive on a side stream while the
            # forward part runs; every copy is inside the timed region
            step.replay_from_host(h_in, h_in["dF"], h_in["color"], h_ups, h_out, h_out["d_dF"], h_out["d_color"])
            torch.cuda.current_stream().synchronize()

        for _ in range(max(3, args.warmup)):
            e2e_step()
        e_steps = max(3, min(args.steps, 20))
        t0 = time.perf_counter()
        for _ in range(e_steps):
            e2e_step()
        ems = (time.perf_counter() - t0) / e_steps * 1e3
        ems = dist.max(ems)
        e2e = {"value": total_px / (ems * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ems,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # ---- the oracle on the host cores (rank 0, one GPU only)
    cpu = None
    if not args.no_cpu and dist.rank == 0 and dist.world == 1:
        import oracle
        v, crop, secs, threads, v_fwd = oracle_sample(scene, 12.0, parts=True)
        # the same oracle on one host thread, on a smaller crop (about 3 s)
        oracle.set_threads(1)
        try:
            v1, crop1, secs1, _, v1_fwd = oracle_sample(scene, 3.0, parts=True)
        finally:
            oracle.set_threads(threads)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"forward+backward of a {crop[2]}x{crop[3]} px crop of view 0 with all "
                         f"{scene.n} splats ({secs:.1f} s)",
               "forward_only": v_fwd,
               "one_thread": {"value": v1, "forward_only": v1_fwd,
                              "sample": f"forward+backward of a {crop1[2]}x{crop1[3]} px crop ({secs1:.1f} s)"}}

    if dist.rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD_TEXT[args.workload], "n_splats": scene.n, "views": len(cams),
                           "main_pixels_per_gpu": main_px, "sun_pixels_per_gpu": sun_px,
                           "storage": args.storage, "tile": f"{opts.tile_w}x{opts.tile_h}",
                           "batch": "{} records per staged batch (forward), {} (backward)".format(*L.staging_batches()),
                           "pixels_per_thread": opts.pixels_per_thread,
                           "launch": "two CUDA graphs per step (forward part, backward part); persistent forward and backward launches over "
                                     "all (target, tile) items",
                           "l2": "not flushed: every step streams > 1 GB of projected records, lists and "
                                 "upstream planes, far above the 129 MB L2",
                           "parallelism": f"replicas x{dist.world}", "intersections": needed,
                           "autotune": tune},
                "roofline": roofline, "cpu_baseline": cpu, "plain_fp32": plain,
                "batched_over_plain": (value / dist.world) / plain["value"] if plain else None,
                "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "clocks": clocks,
                "shade": shade, "depth_normal": dnormal, "distortion": distortion, "optimizer": optimizer,
                "init": init, "single": single, "small": small,
                "steps_per_s": 1e3 / ms_max, "peak_hbm_gb": peak_hbm_gb,
                "device": {"sms": sms, "arch": arch, "name": torch.cuda.get_device_name()}}
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    dist = Dist()
    if args.impl == "reference":
        return run_reference(args, dist)
    return run_ours(args, dist)


if __name__ == "__main__":
    sys.exit(main())
