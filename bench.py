#!/usr/bin/env python
"""Throughput of the BG-Triangle differentiable rasterizer on one node.

Workload (the batched configuration of the metric): 20,000 degree-2
BG-triangles (icosphere + three ellipsoids, control-point noise N(0, 0.02)),
64 views of mixed size {256, 512, 800, 1024}^2 on a radius 3.5..5 sphere,
boundary scale r_b = 1e-2. One step = forward of all 64 views in one batched
call, L1 loss gradient against a fixed target, backward to the primitive
parameters (the metric's fwd+bwd step). Beside it, the training step with
the paper's photometric loss (Eq. 9, L2 + D-SSIM, lambda 0.2) in place of L1. Metric: renders/s, one render = one view forward + backward.
The step's inputs (~0.5 GB of pixels and pairs) exceed the 129 MB L2.

Beside it: the plain single-view path on the same 64 views, one 800^2 view,
an end-to-end number with the parameters copied from pinned host memory and
the gradients read back every step, per-stage device times (CUDA events) for
the roofline of the dominant kernel, SM clocks sampled during the timed
region, and the FP64 CPU oracle timed on a bounded sample of views.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "fwd+bwd renders/s at 800² (20k BG-triangles) batched vs plain; % HBM peak"
WORKLOAD = ("20k degree-2 BG-triangles (icosphere f20 + 3 ellipsoids, noise 0.02), 64 views mixed "
            "{256,512,800,1024}^2, radius U[3.5,5], r_b=1e-2, batched fwd+L1+bwd")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rb", type=float, default=1e-2)
    ap.add_argument("--tile", type=int, default=0, help="0 = autotune")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--sh-degree", type=int, default=0,
                    help="add view-dependent SH colour of this degree (1..3) to the scene")
    ap.add_argument("--attr-res", type=int, default=1,
                    help="rotation / scaling attribute maps of this leg resolution (paper: 3)")
    ap.add_argument("--workload", default="config4",
                    choices=["config4", "view800", "views1024x4", "room8", "views800x64"],
                    help="view800: one 800^2 view of the same scene (small case for profilers); "
                         "room8: the 100k degree-3 room under eight 1600x1200 views (large scale); "
                         "views1024x4: four 1024^2 views (inputs larger than L2, a few GB on the device); "
                         "views800x64: 64 views of 800^2 of the same scene (the metric's resolution, batched)")
    ap.add_argument("--no-rows", action="store_true",
                    help="skip the rows reported beside the headline (r_b = 1e-3, 64 x 800^2 batched vs plain)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, device):
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, views_per_rank, steps, ms):
    """Whole-job renders/s: every rank renders its own views (weak scaling)."""
    return world * views_per_rank * steps / (ms / 1e3)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured", float(d.get("sm_max_mhz", 2070.0))
    except Exception:
        return 6800.0, "fallback", 2070.0


# FP32 peak of a GB300: 152 SMs x 128 FP32 lanes x 2 flop per FMA x SM clock
SMS, FP32_LANES = 152, 128

LAMBDA = 0.2      # weight of the D-SSIM term of Eq. 9
# Algorithmic FP32 operations per pixel and channel of the fused loss: the
# separable 11-tap window over five moments (2 x 5 x 11 FMA) and over three
# SSIM partials (2 x 3 x 11 FMA), SSIM and its partials (~20), the gradient (6)
LOSS_FLOPS_PER_VALUE = 2 * (2 * 5 * 11 + 2 * 3 * 11) + 26

# Algorithmic FP32 operations per work unit of the blending kernels (FMA = 2,
# exp / sqrt / divide = 1): a pair inside a Gaussian's support needs the offset,
# the quadratic form, the exponential, o G and the cutoff test (13); a composited
# pair needs alpha, the transmittance update and three colour FMAs forward (12),
# and the Eq. 6-8 / supplementary chain rule backward (60); one boundary candidate
# of the Eq. 6 search costs a squared distance scaled by 1/sigma^2 and a compare (8).
FLOPS_PER_UNIT = {"support": 13, "fwd_composited": 12, "bwd_composited": 60, "candidate": 8}


def blend_flops(units, which):
    u = units
    if which == "composite_fwd":
        return (FLOPS_PER_UNIT["support"] * u["fwd_support"] + FLOPS_PER_UNIT["fwd_composited"] * u["fwd_composited"]
                + FLOPS_PER_UNIT["candidate"] * u["fwd_candidates"])
    return (FLOPS_PER_UNIT["support"] * u["bwd_support"] + FLOPS_PER_UNIT["bwd_composited"] * u["bwd_composited"]
            + FLOPS_PER_UNIT["candidate"] * u["bwd_candidates"])


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.environ.get("BGT_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), f"bgt_clocks_{os.getpid()}_{index}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() in ("active", "1", "yes"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def stage_bytes(stage, c, M, ncp, V):
    """Algorithmic bytes a stage must move per call (per unit x units)."""
    P, F, Nb, K, Kb = c["P"], c["F"], c["Nb"], c["K"], c["Kb"]
    return {
        # control points per view + one 64-bit depth key per pixel
        "raster": 12 * ncp * M * V + 8 * P,
        # depth key read, I_id + I_uv write
        "resolve": 8 * P + 12 * P,
        # I_id (+ neighbours) and I_uv read, Gaussian (48 B) and boundary (16 B) records written
        "generate": 4 * P + 8 * F + 48 * F + 16 * Nb,
        # pair keys written once, read + written by the per-tile sort
        "binning": 3 * 8 * K + 3 * 8 * Kb + 20 * Kb,
        # per tile: keys + 48-B records of its pairs, 20-B boundary entries; image, T, n, I_id per pixel
        "composite_fwd": 56 * K + 20 * Kb + 12 * P + 8 * P + 4 * P,
        # as forward + dl/dC read + per-Gaussian gradient accumulation (36 B)
        "composite_bwd": 56 * K + 20 * Kb + 12 * P + 12 * P + 36 * F,
        # per-Gaussian / boundary gradients read, parameter gradients written
        "chain": 48 * F + 16 * Nb + 8 * F + 4 * (2 * 3 * ncp + 2) * M,
        "prep": 8 * P,
    }[stage]


# DRAM bytes (read + write) per composited pair of the blending kernels, from one
# ncu capture of four 1024^2 views (profiles/composite_blend_views1024x4.md),
# valid only for the kernel source they were measured on (else traffic: null)
BLEND_TRAFFIC = {"source_sha256": "31926f2fd2cc1a5d3a82528a9d09ede5a53636275ce296cf8d2a83e72afeef5b",
                 "composite_fwd": (131572480 + 153608192) / 50625814,
                 "composite_bwd": (292371712 + 40375552) / 50625814}


# Warp instructions per warp visit of the blending kernels (a visit: one warp,
# one listed Gaussian forward; one replayed record backward), from the same
# capture; the forward keeps the issue slots ~80 % busy, so issue is the
# ceiling that binds it; same source check as the traffic
BLEND_ISSUE = {"source_sha256": BLEND_TRAFFIC["source_sha256"],
               "composite_fwd": 681557800 / 5419084, "composite_bwd": 552831143 / 4948871}


def _blend_source_matches():
    import hashlib
    src = os.path.join(ROOT, "paper_2503_13961_gb300", "csrc", "composite.cu")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return False
    return sha == BLEND_TRAFFIC["source_sha256"]


def blend_traffic(dom, units):
    if not _blend_source_matches() or dom not in BLEND_TRAFFIC:
        return None
    pairs = units["fwd_composited" if dom == "composite_fwd" else "bwd_composited"]
    return int(BLEND_TRAFFIC[dom] * pairs)


def blend_issue(dom, units, ms, sm_mhz):
    """Instruction-issue view of a blending kernel: warp instructions per launch
    (captured per warp visit, scaled by this run's visits) over the live
    duration, against 152 SMs x 4 schedulers x 1 warp instruction per cycle."""
    if not _blend_source_matches() or dom not in BLEND_ISSUE:
        return None
    visits = units["fwd_warp_visits" if dom == "composite_fwd" else "bwd_warp_visits"]
    instr = BLEND_ISSUE[dom] * visits
    peak = SMS * 4 * sm_mhz * 1e6
    ach = instr / (ms * 1e-3)
    return {"achieved": round(ach / 1e12, 4), "peak": round(peak / 1e12, 4), "unit": "T warp-instr/s",
            "frac": round(ach / peak, 4), "warp_instr_per_launch": int(instr),
            "peak_kind": "derived: 152 SMs x 4 schedulers x 1 instruction per cycle x max SM clock"}


def roofline_entry(dom, stage_ms, units, achieved_gbs, dom_bytes, peak, peak_kind, fp32_peak, sm_mhz):
    """Roofline of the dominant kernel: the blending kernels are bound by FP32
    issue (no dense contraction, DRAM far from busy), the others by HBM."""
    ms = stage_ms[dom]
    if dom in ("composite_fwd", "composite_bwd") and units:
        fl = blend_flops(units, dom)
        ach = fl / (ms * 1e-3) / 1e12
        return {"bound": "alu", "kernel": dom, "achieved": round(ach, 3), "peak": round(fp32_peak, 1),
                "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock", "unit": "TFLOP/s",
                "frac": round(ach / fp32_peak, 4), "traffic": blend_traffic(dom, units), "alg_flops_per_launch": int(fl),
                "ms_per_launch": round(ms, 4),
                "hbm_view": {"achieved": round(achieved_gbs, 1), "peak": peak, "unit": "GB/s",
                             "frac": round(achieved_gbs / peak, 4), "alg_bytes_per_launch": int(dom_bytes)},
                "issue_view": blend_issue(dom, units, ms, sm_mhz)}
    return {"bound": "hbm", "kernel": dom, "achieved": round(achieved_gbs, 1), "peak": peak, "peak_kind": peak_kind,
            "unit": "GB/s", "frac": round(achieved_gbs / peak, 4), "traffic": None,
            "alg_bytes_per_launch": int(dom_bytes), "ms_per_launch": round(ms, 4)}


def build_workload(seed_views, rb, workload="config4", sh_degree=0, attr_res=1):
    from paper_2503_13961_gb300 import scenes
    if workload == "room8":
        return scenes.config_scene(5, r_b=rb)[:2]
    sc, cams = scenes.config_scene(4, r_b=rb)
    if attr_res > 1:
        sc = scenes.with_attribute_maps(sc, attr_res)
    if sh_degree > 0:
        sc = scenes.with_sh(sc, sh_degree)
    if workload == "view800":
        return sc, [c for c in cams if c["width"] == 800][:1]
    if workload == "views1024x4":
        return sc, [c for c in cams if c["width"] == 1024][:4]
    if workload == "views800x64":
        return sc, views800x64(seed_views)
    if seed_views:
        # other ranks render their own 64 views of the same scene (weak scaling)
        rng = np.random.default_rng(1000 + seed_views)
        sizes = [(c["width"], c["height"]) for c in cams]
        cams = scenes.make_views(rng, sizes, 3.5, 5.0)
    return sc, cams


def workload_name(workload, rb=1e-2):
    if workload == "room8":
        return ("100k degree-3 BG-triangles (10^3 room of 19,200 + 100 cubes + 100 spheres, noise 0.01, "
                "opacity Beta(5,1)), eight 1600x1200 views, batched fwd+L1+bwd")
    return {"config4": "", "view800": "one 800^2 view of: ", "views1024x4": "four 1024^2 views of: ",
            "views800x64": "64 views of 800^2 (radius U[3.5,5]) of: "}[workload] + WORKLOAD.replace(
                "r_b=1e-2", f"r_b={rb:g}")


def views800x64(seed=0):
    """64 views of 800^2 of the config-4 scene, directions uniform on S^2,
    radius U[3.5, 5] (the metric's resolution at the batch size of config 4)."""
    from paper_2503_13961_gb300 import scenes
    rng = np.random.default_rng(800 + seed)
    return scenes.make_views(rng, [(800, 800)] * 64, 3.5, 5.0)


def time_batched(R, sc, cams, tuning, steps, stream, ppp=6, plain=False):
    """renders/s of the batched fwd + L1 + bwd step on `cams` (graph, one
    handle for all views), or of the plain single-view path (one call per
    view) with plain=True; CUDA events on `stream` after 3 warm-up steps."""
    import torch
    dev = R.scene_to_device(sc)
    M = sc["ctrl"].shape[0]
    sizes = [c["width"] * c["height"] for c in cams]
    P = sum(sizes)
    cap = max(sizes) if plain else P
    rd = R.Renderer(degree=int(sc["degree"]), max_prims=M, max_views=1 if plain else len(cams), max_pixels=cap,
                    max_pairs=ppp * cap, max_boundary_pairs=ppp * cap, graph=not plain)
    rd.set_tuning(**tuning)
    gen = torch.Generator(device="cuda").manual_seed(4321)
    with torch.cuda.stream(stream):
        images = torch.empty((P, 3), device="cuda")
        target = torch.rand((P, 3), device="cuda", generator=gen)
        dimg = torch.zeros((P, 3), device="cuda")
        grads = {k: torch.empty_like(dev[k]) for k in R.GRAD_KEYS if k in dev}
    torch.cuda.synchronize()
    offs = np.concatenate([[0], np.cumsum(sizes)])
    ccams = R.Cameras(cams)
    one = [R.Cameras([c]) for c in cams]

    def step():
        if plain:
            for v in range(len(cams)):
                a, b = int(offs[v]), int(offs[v + 1])
                rd.forward(dev, one[v], images[a:b], stream=stream)
                rd.l1_loss_grad(images[a:b], target[a:b], 1.0 / (3 * (b - a)), dimg[a:b], stream=stream)
                rd.backward(dev, one[v], dimg[a:b], grads, stream=stream)
        else:
            rd.forward(dev, ccams, images, stream=stream)
            rd.l1_loss_grad(images, target, 1.0 / (3 * P), dimg, stream=stream)
            rd.backward(dev, ccams, dimg, grads, stream=stream)

    for _ in range(3):
        step()
    rd.sync_status(stream)
    counts = rd.counts(stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    rd.sync_status(stream)
    rd.close()
    return {"value": round(len(cams) / (ms * 1e-3), 2), "unit": "renders/s", "ms_per_step": round(ms, 4),
            "views": len(cams), "pixels": int(P), "tuning": tuning, "graph": not plain,
            "counts": {k: int(v) for k, v in counts.items()}}


def run_rows(args, tuning, stream):
    """Rows reported beside the headline: the batched step at the paper's
    other boundary scale r_b = 1e-3 (Table 4), and 64 views of 800^2 (the
    metric's resolution) batched against the plain single-view path."""
    from paper_2503_13961_gb300 import render as R
    from paper_2503_13961_gb300 import scenes
    steps = max(3, min(args.steps, 10))
    sc3, cams3 = scenes.config_scene(4, r_b=1e-3)
    rows = {"rb_1e-3": time_batched(R, sc3, cams3, tuning, steps, stream)}
    rows["rb_1e-3"]["workload"] = WORKLOAD.replace("r_b=1e-2", "r_b=1e-3")
    sc, _ = scenes.config_scene(4, r_b=args.rb)
    c800 = views800x64()
    b = time_batched(R, sc, c800, tuning, steps, stream)
    pl = time_batched(R, sc, c800, dict(tuning, tile_size=16), max(2, steps // 2), stream, plain=True)
    b["workload"] = pl["workload"] = "64 views of 800^2 of the config-4 scene (radius U[3.5,5]), fwd+L1+bwd"
    rows["batched_800x64"] = b
    rows["plain_800x64"] = pl
    rows["batched_over_plain_800x64"] = round(b["value"] / pl["value"], 3)
    return rows


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2503_13961_gb300 import render as R

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sc, cams = build_workload(rank, args.rb, args.workload, args.sh_degree, args.attr_res)
    cams = R.Cameras(cams)  # the C camera array is built once for the whole run
    V = len(cams)
    P = sum(c["width"] * c["height"] for c in cams)
    M, ncp = sc["ctrl"].shape[0], sc["ctrl"].shape[1]
    n = int(sc["degree"])
    ppp = 32 if args.workload == "room8" else 6  # pair capacity per pixel (the room is dense)
    bpp = 24 if args.workload == "room8" else 0   # blend records per pixel (0: the default, 8)
    rd = R.Renderer(degree=n, max_prims=M, max_views=V, max_pixels=P, max_pairs=ppp * P, max_boundary_pairs=ppp * P,
                    max_blend_pairs=bpp * P, tile_size=16, graph=True)
    dev = R.scene_to_device(sc)
    stream = torch.cuda.Stream()
    gen = torch.Generator(device="cuda").manual_seed(1234 + rank)
    with torch.cuda.stream(stream):
        images = torch.empty((P, 3), device="cuda")
        target = torch.rand((P, 3), device="cuda", generator=gen)
        dimg = torch.zeros((P, 3), device="cuda")
        grads = {k: torch.empty_like(dev[k]) for k in R.GRAD_KEYS if k in dev}
        loss = torch.zeros(1, device="cuda")
    torch.cuda.synchronize()  # scene tensors were filled on the default stream
    scale = 1.0 / (3 * P)
    tune_ms = None
    if args.tile:
        rd.set_tile_size(args.tile)
    else:
        # the tuner times the step's backward with the L1 gradient of one
        # forward (zero gradients would skip the backward's atomics); 5 passes
        # per candidate: the knobs differ by 1-3 %
        with torch.cuda.stream(stream):
            rd.forward(dev, cams, images, stream=stream)
            rd.l1_loss_grad(images, target, scale, dimg, torch.zeros(1, device="cuda"), stream=stream)
        _, tune_ms = rd.autotune(dev, cams, images, dimg, grads, iters=5, stream=stream)

    def step():
        rd.forward(dev, cams, images, stream=stream)
        rd.l1_loss_grad(images, target, scale, dimg, loss, stream=stream)
        rd.backward(dev, cams, dimg, grads, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    rd.sync_status(stream)
    counts = rd.counts(stream)
    counts["P"] = P
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    e1.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    torch.cuda.synchronize()
    if world > 1:
        ms = max_over_ranks(ms, "cuda")
        dist.barrier()
    rd.sync_status(stream)
    value = job_value(world, V, args.steps, ms)

    # per-stage device time of the same step: a second handle (no graph, same
    # scheduling) records CUDA events between the stages on the same stream,
    # timing the step's own kernels; one more pass with the blending kernels'
    # counting build gives their work units
    prof_rd = R.Renderer(degree=n, max_prims=M, max_views=V, max_pixels=P, max_pairs=ppp * P,
                         max_boundary_pairs=ppp * P, max_blend_pairs=bpp * P, tile_size=rd.tile_size, graph=False)
    prof_rd.set_tuning(**rd.tuning())
    stage_ms = {}
    units = {}
    nprof = max(3, min(args.steps, 8))

    def prof_pass():
        prof_rd.forward(dev, cams, images, stream=stream)
        prof_rd.l1_loss_grad(images, target, scale, dimg, loss, stream=stream)
        prof_rd.backward(dev, cams, dimg, grads, stream=stream)
        stream.synchronize()
        return prof_rd.profile()

    prof_rd.set_profiling(True, count_units=True)
    _, _, _, units = prof_pass()
    prof_rd.set_profiling(True, count_units=False)
    for i in range(nprof + 1):
        prof, kf, kb, _ = prof_pass()
        if i == 0:
            continue  # warm-up
        for k, v in prof.items():
            stage_ms[k] = stage_ms.get(k, 0.0) + v / nprof
    prof_rd.sync_status(stream)
    prof_rd.close()
    del prof_rd
    launches_per_step = kf + kb + 1  # + the L1 loss-gradient kernel

    # end to end: parameters from pinned host memory in, gradients + loss out, every step
    host_in = {k: dev[k].cpu().pin_memory() for k in R.SCENE_KEYS}
    host_out = {k: torch.empty(grads[k].shape, dtype=torch.float32).pin_memory() for k in grads}
    host_loss = torch.empty(1).pin_memory()
    h2d = sum(t.numel() * 4 for t in host_in.values())
    d2h = sum(t.numel() * 4 for t in host_out.values()) + 4

    def e2e_step():
        for k in R.SCENE_KEYS:
            dev[k].copy_(host_in[k], non_blocking=True)
        step()
        for k in grads:
            host_out[k].copy_(grads[k], non_blocking=True)
        host_loss.copy_(loss, non_blocking=True)

    with torch.cuda.stream(stream):
        for _ in range(2):
            e2e_step()
        stream.synchronize()
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        e1.synchronize()
        wall = time.perf_counter() - t0
    e2e_ms = max(e0.elapsed_time(e1), wall * 1e3)
    if world > 1:
        e2e_ms = max_over_ranks(e2e_ms, "cuda")
    e2e_value = job_value(world, V, args.steps, e2e_ms)
    rd.sync_status(stream)

    out = None
    if rank == 0:
        dom = max(("composite_fwd", "composite_bwd", "raster", "generate", "binning", "chain", "resolve"),
                  key=lambda s: stage_ms.get(s, 0.0))
        peak, peak_kind, sm_mhz = peaks()
        fp32_peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
        per_stage = {}
        for s_name, s_ms in stage_ms.items():
            b = stage_bytes(s_name, counts, M, ncp, V)
            per_stage[s_name] = {"ms": round(s_ms, 4), "alg_bytes": int(b),
                                 "GBps": round(b / (s_ms * 1e-3) / 1e9, 1) if s_ms > 0 else None,
                                 "hbm_frac": round(b / (s_ms * 1e-3) / 1e9 / peak, 4) if s_ms > 0 else None}
            if s_name in ("composite_fwd", "composite_bwd") and units:
                fl = blend_flops(units, s_name)
                per_stage[s_name]["alg_flops"] = int(fl)
                per_stage[s_name]["TFLOPs"] = round(fl / (s_ms * 1e-3) / 1e12, 3)
                per_stage[s_name]["alu_frac"] = round(fl / (s_ms * 1e-3) / 1e12 / fp32_peak, 4)
        dom_bytes = stage_bytes(dom, counts, M, ncp, V)
        achieved = dom_bytes / (stage_ms[dom] * 1e-3) / 1e9
        out = {
            "metric": METRIC, "value": round(value, 2), "unit": "renders/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded scene generator; stands in for Lego / NeRF-Synthetic)",
            "config": {"workload": workload_name(args.workload, args.rb),
                       "views": V, "pixels": P, "prims": M, "degree": n,
                       "sh_degree": args.sh_degree, "attr_res": args.attr_res,
                       "tile": rd.tile_size, "tile_autotune_ms": tune_ms, "tuning": rd.tuning(), "graph": True,
                       "counts": {k: int(v) for k, v in counts.items()},
                       "l2": "inputs larger than L2 (no flush needed)", "parallelism": f"replicas x{world}"},
            "clocks": clk,
            "e2e": {"value": round(e2e_value, 2), "unit": "renders/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches_per_step * args.steps),
            "roofline": roofline_entry(dom, stage_ms, units, achieved, dom_bytes, peak, peak_kind, fp32_peak, sm_mhz),
            "work_units": units,
            "stages": per_stage,
        }
    if rank == 0:
        out["train_step_eq9"] = run_eq9_step((rd, dev, cams, sc, stream), images, target, dimg, grads, args)
        out["split_prune"] = run_split_prune((rd, dev, cams, sc, stream), grads)
        if args.workload == "config4" and world == 1 and not args.no_rows:
            out["rows"] = run_rows(args, rd.tuning(), stream)
    return out, (rd, dev, cams, sc, stream)


def run_eq9_step(rd_ctx, images, target, dimg, grads, args):
    """The training step with the paper's photometric loss (Eq. 9, L2 +
    D-SSIM, lambda 0.2) in place of L1: renders/s of forward + loss +
    backward, and the loss kernel alone (CUDA events, roofline figures)."""
    import torch
    rd, dev, cams, _, stream = rd_ctx
    V = len(cams)
    P = images.shape[0]
    loss = torch.zeros(1, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step():
        rd.forward(dev, cams, images, stream=stream)
        loss.zero_()
        rd.l2_dssim_loss_grad(images, target, cams, LAMBDA, 1.0 / V, dimg, loss, stream=stream)
        rd.backward(dev, cams, dimg, grads, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(3):
            step()
        steps = max(3, args.steps)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        for _ in range(3):
            rd.l2_dssim_loss_grad(images, target, cams, LAMBDA, 1.0 / V, dimg, loss, stream=stream)
        e0.record(stream)
        for _ in range(10):
            rd.l2_dssim_loss_grad(images, target, cams, LAMBDA, 1.0 / V, dimg, loss, stream=stream)
        e1.record(stream)
        e1.synchronize()
        lms = e0.elapsed_time(e1) / 10
    rd.sync_status(stream)
    peak, _, sm_mhz = peaks()
    fp32_peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    fl = LOSS_FLOPS_PER_VALUE * 3 * P
    return {"value": round(V / (ms * 1e-3), 2), "unit": "renders/s", "ms_per_step": round(ms, 4),
            "loss_kernel": {"ms": round(lms, 4), "alg_bytes": 36 * P, "alg_flops": int(fl),
                            "TFLOPs": round(fl / (lms * 1e-3) / 1e12, 3),
                            "alu_frac": round(fl / (lms * 1e-3) / 1e12 / fp32_peak, 4),
                            "hbm_frac": round(36 * P / (lms * 1e-3) / 1e9 / peak, 4)}}


def run_split_prune(rd_ctx, grads):
    """Splitting / pruning on the workload's primitives (Sec. 3.3): the
    visibility measures of the step's views, the per-primitive measures and
    flags with the step's control-point gradients, and the 1 -> 4 split of
    every primitive; CUDA-event times and the HBM fraction of their
    algorithmic bytes."""
    import torch
    from paper_2503_13961_gb300 import render as R
    _, dev, _, sc, stream = rd_ctx
    M, ncp = sc["ctrl"].shape[0], sc["ctrl"].shape[1]
    T = int(dev.get("attr_res", 1)) * (int(dev.get("attr_res", 1)) + 1) // 2
    sel = torch.arange(M, dtype=torch.int32, device="cuda")
    peak, _, _ = peaks()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    # algorithmic bytes: metrics read ctrl + gradient and write 13 B per primitive;
    # the split reads the parent's control points, colours and attributes and
    # writes four pieces
    rd = rd_ctx[0]
    P = sum(c["width"] * c["height"] for c in rd_ctx[2])
    vc = torch.zeros(M, dtype=torch.int32, device="cuda")
    cm = torch.zeros((M, 2), dtype=torch.int64, device="cuda")
    cams = rd_ctx[2]
    train = torch.rand((P, 3), device="cuda", generator=torch.Generator(device="cuda").manual_seed(77))
    edges = torch.empty(P, device="cuda")
    es = torch.zeros(M, device="cuda")
    ec = torch.zeros(M, dtype=torch.int32, device="cuda")
    work = {
        # the last forward's I_id and depth keys read, per-primitive counts and masks updated
        "visibility": (lambda: rd.visibility(M, vc, cm, stream=stream), 12 * P + 24 * M),
        # training image read (3 floats per pixel), edge magnitude written
        "edge_magnitude": (lambda: R.edge_magnitude(train, cams, edges, stream=stream), 16 * P),
        # edge magnitude and I_id read, per-primitive sums and counts updated
        "edge_prior": (lambda: rd.edge_prior(edges, M, es, ec, stream=stream), 8 * P + 16 * M),
        "prim_metrics": (lambda: R.prim_metrics(dev, grads["ctrl"], stream=stream), M * (24 * ncp + 13)),
        "subdivide": (lambda: R.subdivide(dev, sel, stream=stream),
                      M * (4 + 24 * ncp + 8 + 28 * T) + 4 * M * (24 * ncp + 8 + 28 * T)),
    }
    with torch.cuda.stream(stream):
        for name, (fn, nbytes) in work.items():
            for _ in range(3):
                fn()
            reps = 20
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            res[name] = {"ms": round(ms, 4), "alg_bytes": int(nbytes),
                         "GBps": round(nbytes / (ms * 1e-3) / 1e9, 1),
                         "hbm_frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4)}
    res["prims"] = M
    return res


def run_plain(rd_ctx, args):
    """The single-view path: each view rendered and differentiated on its own."""
    import torch
    from paper_2503_13961_gb300 import render as R
    _, dev, cams, sc, stream = rd_ctx
    M = sc["ctrl"].shape[0]
    Pmax = max(c["width"] * c["height"] for c in cams)
    ppp = 32 if args.workload == "room8" else 6
    bpp = 24 if args.workload == "room8" else 0
    rd = R.Renderer(degree=int(sc["degree"]), max_prims=M, max_views=1, max_pixels=Pmax, max_pairs=ppp * Pmax,
                    max_boundary_pairs=ppp * Pmax, max_blend_pairs=bpp * Pmax, tile_size=16, graph=False)
    bufs = []
    gen = torch.Generator(device="cuda").manual_seed(99)
    with torch.cuda.stream(stream):
        for c in cams:
            n = c["width"] * c["height"]
            bufs.append((torch.empty((n, 3), device="cuda"), torch.rand((n, 3), device="cuda", generator=gen),
                         torch.zeros((n, 3), device="cuda")))
        grads = {k: torch.empty_like(dev[k]) for k in R.GRAD_KEYS if k in dev}

    def step():
        for c, (img, tgt, d) in zip(cams, bufs):
            rd.forward(dev, [c], img, stream=stream)
            rd.l1_loss_grad(img, tgt, 1.0 / img.numel(), d, stream=stream)
            rd.backward(dev, [c], d, grads, stream=stream)

    step()
    rd.sync_status(stream)
    steps = max(2, args.steps // 2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    rd.sync_status(stream)
    plain = {"value": round(len(cams) * steps / (ms / 1e3), 2), "unit": "renders/s",
             "ms_per_64_views": round(ms / steps, 3), "graph": False, "tile": 16}
    # one 800^2 view, plain
    i800 = [i for i, c in enumerate(cams) if c["width"] == 800][:1]
    c800 = [cams[i] for i in i800]
    v800 = None
    if c800:
        img, tgt, d = bufs[i800[0]]
        for _ in range(3):
            rd.forward(dev, c800, img, stream=stream)
            rd.l1_loss_grad(img, tgt, 1.0 / img.numel(), d, stream=stream)
            rd.backward(dev, c800, d, grads, stream=stream)
        n = 20
        e0.record(stream)
        for _ in range(n):
            rd.forward(dev, c800, img, stream=stream)
            rd.l1_loss_grad(img, tgt, 1.0 / img.numel(), d, stream=stream)
            rd.backward(dev, c800, d, grads, stream=stream)
        e1.record(stream)
        e1.synchronize()
        v800 = {"value": round(n / (e0.elapsed_time(e1) / 1e3), 2), "unit": "renders/s",
                "ms_per_render": round(e0.elapsed_time(e1) / n, 4)}
    rd.close()
    return plain, v800


def sample_views(cams):
    """The CPU sample of a mixed-size workload: the first view of each size
    (256, 512, 800 and 1024 squared in config 4), largest first, so that
    every resolution of the mix is timed."""
    first = {}
    for i, c in enumerate(cams):
        first.setdefault((c["width"], c["height"]), i)
    return sorted(first.values(), key=lambda i: -cams[i]["width"] * cams[i]["height"])


def oracle_views(sc, cams, idx, rng):
    """Forward, L1 loss gradient and backward of the views `idx` with the FP64
    oracle; returns the pixels processed."""
    from oracle import oracle
    pix = 0
    for i in idx:
        c = cams[i]
        idm, uv, _ = oracle.raster(sc, c)
        img = oracle.render(sc, c, idm, uv)["image"]
        gt = rng.uniform(size=img.shape)
        dl = np.sign(img - gt) / img.size  # the L1 loss gradient of the GPU step
        oracle.backward(sc, c, dl, idm, uv)
        pix += c["width"] * c["height"]
    return pix


def cpu_workload(rb, sh_degree=0, attr_res=1):
    from paper_2503_13961_gb300 import scenes
    sc, cams = scenes.config_scene(4, r_b=rb)
    if attr_res > 1:
        sc = scenes.with_attribute_maps(sc, attr_res)
    if sh_degree > 0:
        sc = scenes.with_sh(sc, sh_degree)
    return sc, cams


def sample_text(cams, idx, passes, dt):
    names = ", ".join(f"#{i} ({cams[i]['width']}^2)" for i in idx)
    return (f"{passes} pass(es) over views {names} of the 64-view workload (one view of each size), "
            f"fwd+L1+bwd, FP64, {dt:.1f} s")


def cpu_baseline(budget_s, rb, sh_degree=0, attr_res=1):
    """The FP64 oracle on the host cores: passes over the stratified sample of
    the workload (one view of each size) until the time budget is used;
    renders/s and pixels/s."""
    from oracle import oracle
    sc, cams = cpu_workload(rb, sh_degree, attr_res)
    idx = sample_views(cams)
    rng = np.random.default_rng(0)
    passes, t0, pix = 0, time.perf_counter(), 0
    while True:
        pix += oracle_views(sc, cams, idx, rng)
        passes += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": round(passes * len(idx) / dt, 4), "unit": "renders/s", "cores": oracle.num_threads(),
            "kind": "oracle", "pixels_per_s": round(pix / dt, 1), "sample": sample_text(cams, idx, passes, dt)}


def run_reference(args, world):
    """The reference arm: the FP64 oracle (the paper publishes no code), each
    step one pass over the same stratified sample as cpu_baseline."""
    from oracle import oracle
    oracle.build()
    sc, cams = cpu_workload(args.rb, args.sh_degree, args.attr_res)
    idx = sample_views(cams)
    rng = np.random.default_rng(0)
    for _ in range(args.warmup):
        oracle_views(sc, cams, idx[-1:], rng)  # the smallest view: page in, spawn the thread pool
    t0 = time.perf_counter()
    pix = 0
    for _ in range(args.steps):
        pix += oracle_views(sc, cams, idx, rng)
    dt = time.perf_counter() - t0
    val = args.steps * len(idx) / dt
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": "renders/s",
                      "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": round(dt * 1e3 / max(args.steps, 1), 2),
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": workload_name("config4", args.rb)},
                      "cpu_baseline": {"kind": "oracle", "cores": oracle.num_threads(),
                                       "sample": sample_text(cams, idx, args.steps, dt),
                                       "value": round(val, 4), "unit": "renders/s",
                                       "pixels_per_s": round(pix / dt, 1)},
                      "e2e": {"value": round(val, 4), "unit": "renders/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def main():
    args = parse()
    world, rank, _ = dist_env()
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, world)
        return
    out, ctx = run_ours(args)
    if rank == 0:
        if world == 1 and not args.no_plain:
            plain, v800 = run_plain(ctx, args)
            out["plain"] = plain
            out["batched_over_plain"] = round(out["value"] / plain["value"], 3)
            out["view_800"] = v800
        if world == 1:
            out["cpu_baseline"] = cpu_baseline(args.cpu_seconds, args.rb, args.sh_degree, args.attr_res)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
