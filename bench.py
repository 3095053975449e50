#!/usr/bin/env python
"""Benchmark of the 2DGS rasterizer forward + backward (the refinement step
of Flash-Mono's mapping backend) on synthetic indoor submaps.

Default workload: one submap of 32 keyframes x 512x384 per-pixel surfels
(6,291,456 surfels) along a seeded trajectory through a 3-room layout,
rendered forward and backward from all 32 keyframe poses at 512x384.  One
step = preprocess + bin/sort + forward compositing + tile adjoint + chain
rule to surfel parameters and per-view poses, for all 32 views (the upstream
gradient is the L1 RGB + 0.1 L1 depth loss gradient against the keyframes'
ray-cast targets, computed once before timing).

Prints one JSON line (see the end of main()).  Under torchrun each rank
renders its own independent submap (weak scaling, no collective on the
data path); rank 0 prints the max-over-ranks timing.

--impl reference times the FP64 CPU oracle (the reference statement of the
method) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2DGS raster fwd+bwd ms/view & views/s at 6.3M surfels; fraction of roofline"
FP32_LANES_PER_SM = 128   # FP32 lanes per SM (4 sub-partitions x 32)
MUFU_LANES_PER_SM = 16    # special-function (ex2, rcp) results per SM per clock

# Algorithmic work per unit of each stage, as the method defines it (the
# counts the kernels report times these figures; nothing here is measured):
#   compositing forward, per processed (pixel, surfel) pair -- every entry up
#   to the pixel's stop whose rect holds the pixel, skipped or blended: about
#   32 FP32 lane-instructions and 2 special-function ops (rcp, ex2); per
#   instance the 4-byte list entry and the 76-byte record read once; per
#   pixel 40 bytes of outputs and per-pixel state written.
#   compositing backward, per processed pair: about 100 FP32
#   lane-instructions and 3 special-function ops; per instance the 80-byte
#   record read once; per pixel 72 bytes of upstream gradient and state
#   read; per visible (view, surfel) its 80-byte gradient record written.
INSTR_FWD, MUFU_FWD = 32, 2
INSTR_BWD, MUFU_BWD = 100, 3
FWD_BYTES_INST, FWD_BYTES_PIX = 80, 40
BWD_BYTES_INST, BWD_BYTES_PIX, BWD_BYTES_VIS = 80, 72, 80
# the same figures as reported with the roofline's kernel ("pair" = processed pair)
PER_UNIT = {
    "render_fwd": {"instr_per_pair": INSTR_FWD, "mufu_per_pair": MUFU_FWD, "bytes_per_instance": FWD_BYTES_INST,
                   "bytes_per_pixel": FWD_BYTES_PIX},
    "render_bwd": {"instr_per_pair": INSTR_BWD, "mufu_per_pair": MUFU_BWD, "bytes_per_instance": BWD_BYTES_INST,
                   "bytes_per_pixel": BWD_BYTES_PIX, "bytes_per_visible": BWD_BYTES_VIS},
}

# The same kernels' own FP32 arithmetic per pair, counted from their source
# (an FMA counts 2), reported beside the figures above:
#   alpha of a pair 29 FLOP; blend of a kept pair 18; reverse of a kept pair 63.
FLOP_EVAL = 29
FLOP_BLEND = 18
FLOP_BWD = 63


def _workloads():
    from paper_2604_03092_gb300 import scenes
    return {
        "submap32": ("32 keyframes x 512x384 = 6,291,456 surfels, 32 views at 512x384 (fx=fy=400), 3-room layout",
                     lambda seed: scenes.submap_scene(seed=2001 + seed)),
        "submap8": ("8 keyframes x 512x384 = 1,572,864 surfels, 8 views at 512x384 (a smaller submap for profiling)",
                    lambda seed: scenes.submap_scene(seed=2001 + seed, n_keyframes=8)),
        "keyframe8": ("one 512x384 keyframe = 196,608 surfels, 8 perturbed views at 512x384",
                      lambda seed: scenes.keyframe_scene(seed=1001 + seed)),
        "random4096": ("4,096 random surfels, one 128x96 view",
                       lambda seed: scenes.random_scene(n=4096, seed=seed)),
        "uneven64": ("64 submaps, log-uniform [50k, 2M] surfels, images from {320x240, 512x384, 640x480}, 4 views each",
                     lambda seed: scenes.uneven_batch_scene(seed=3001 + seed)),
        "largemap150": ("150 keyframes x 512x384 = 29,491,200 surfels, 6 rooms, 16 views at 640x480 (fx=fy=500)",
                        lambda seed: scenes.large_map_scene(seed=4001 + seed)),
    }


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"splat2d_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.uuid:
                cmd[1:1] = ["-i", self.uuid]
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self) -> dict:
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            d["source"] = "measured"
            return d
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "source": "fallback"}


# ---------------------------------------------------------------------------
# the oracle on the host cores (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_views(sc, views, seed: int = 0):
    """Time the FP64 oracle, as it stands, on whole views of the workload:
    per view the preprocess of its surfel range, the forward at every pixel
    and the reverse pass at every pixel (seeded upstream gradient) with the
    chain rule.  Returns (seconds per view, description, wall seconds)."""
    import oracle
    cfg = oracle.Config(tile_w=16, tile_h=16)
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    for v in views:
        H, W = sc.views[v].height, sc.views[v].width
        p = oracle.preprocess_scene_view(sc, v, cfg)
        oracle.render(p)
        off, cnt = sc.view_ranges()[v]
        sl = slice(off, off + cnt)
        oracle.render_bwd(sc.means[sl], sc.scales[sl], sc.quats[sl], p, rng.normal(size=(8, H, W)))
    wall = time.perf_counter() - t0
    desc = (f"views {list(views)} of the workload, each in full: oracle preprocess of the view's surfels, forward "
            f"and reverse pass at every pixel, chain rule (measured {wall:.1f} s on {_omp_threads()} threads)")
    return wall / len(views), desc, wall


def oracle_timing_child():
    """Child-process body of `oracle_timing` (OpenMP fixes its thread count
    at load): prints one JSON object with the seconds the oracle takes, as it
    stands, for the forward and reverse pass (with the chain rule) of the
    4,096-surfel random scene in definition mode (every surfel at every
    pixel) and of all 8 views of the 512x384 keyframe workload (binned)."""
    import oracle
    from paper_2604_03092_gb300 import scenes

    def fb(sc, v, mode, cfg):
        H, W = sc.views[v].height, sc.views[v].width
        p = oracle.preprocess_scene_view(sc, v, cfg)
        oracle.render(p, mode)
        off, cnt = sc.view_ranges()[v]
        sl = slice(off, off + cnt)
        up = np.random.default_rng(v).normal(size=(8, H, W))
        oracle.render_bwd(sc.means[sl], sc.scales[sl], sc.quats[sl], p, up, mode=mode)
    sc0 = scenes.random_scene(n=4096, seed=0)
    t0 = time.perf_counter()
    fb(sc0, 0, 0, oracle.Config())
    t_def = time.perf_counter() - t0
    sc1 = scenes.keyframe_scene(seed=1001)
    t0 = time.perf_counter()
    for v in range(len(sc1.views)):
        fb(sc1, v, 1, oracle.Config(tile_w=8, tile_h=8))
    t_kf = time.perf_counter() - t0
    print(json.dumps({"random4096_definition_s": t_def, "keyframe8_all_views_s": t_kf,
                      "threads": _omp_threads()}), flush=True)


def oracle_timing() -> dict:
    """The oracle's breadth timings, 1 thread and all host cores (child
    processes): definition mode on the 4,096-surfel scene, and the 8-view
    512x384 keyframe workload.  About 20 s in all."""
    res = {}
    for label, threads in (("threads_1", 1), ("threads_all", os.cpu_count() or 1)):
        env = dict(os.environ, OMP_NUM_THREADS=str(threads))
        r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-timing-child"], env=env,
                           capture_output=True, text=True, timeout=600)
        try:
            res[label] = json.loads(r.stdout.strip().splitlines()[-1])
        except (ValueError, IndexError):
            res[label] = {"failed": r.stderr[-300:]}
    return res


def _omp_threads() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def _config(args, wl_desc, sc, world):
    """The workload's description, identical in both arms' lines."""
    return {"workload": args.workload, "description": wl_desc, "views": len(sc.views), "surfels": sc.n,
            "l2": "inputs larger than L2 (records + instances > 129 MB)",
            "parallelism": f"{world} independent submap(s), one per GPU"}


def run_reference(args, wl_desc, make):
    """The oracle on the host cores.  One step renders one whole view of the
    workload (its preprocess, the forward and reverse pass at every pixel and
    the chain rule; views in turn), so ms_per_step is the measured time of
    one such step and value the views per second it sustains."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sc = make(0)
    times, descs = [], []
    for i in range(args.warmup + args.steps):
        per_view, desc, wall = oracle_views(sc, [i % len(sc.views)], seed=i)
        if i >= args.warmup:
            times.append(per_view)
            descs.append(i % len(sc.views))
    per_step = float(np.mean(times))
    value = 1.0 / per_step
    sample = (f"one whole view of the {len(sc.views)}-view workload per step (views {descs} in turn): oracle "
              f"preprocess of the view's surfels, forward and reverse pass at every pixel, chain rule; "
              f"{_omp_threads()} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "views/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "views_per_step": 1,
        "ms_per_view": per_step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": _config(args, wl_desc, sc, args.gpus),
        "cpu_baseline": {"value": value, "unit": "views/s", "cores": _omp_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "views/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------
STAGE_SOURCE = {"render_bwd": "render.cu", "render_fwd": "render.cu", "preprocess": "preprocess.cu",
                "preprocess_bwd": "preprocess.cu", "bin_sort": "binsort.cu"}


def _recorded_traffic(stage: str, cfg, n_inst: int):
    """DRAM bytes per launch of the stage's kernel at this launch's
    instance count, scaled from the ncu capture recorded on the smaller
    8-keyframe submap (profiles/traffic_<kernel>_submap8.txt: captures that
    hold a few GB on the device) by the ratio of instances, which is what the
    compositing kernels' traffic grows with; None unless the capture was
    taken on the current kernel source (sha256 of its .cu file) and launch
    shape."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"traffic_k_{stage}_submap8.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#") and " " in line:
            k, v = line.split(None, 1)
            rec[k] = v
    src = os.path.join(ROOT, "paper_2604_03092_gb300", "csrc", STAGE_SOURCE.get(stage, ""))
    if rec.get("stage") != stage or not os.path.isfile(src):
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != rec.get("source_sha256"):
        return None
    shape = f"{cfg.tile_w}x{cfg.tile_h}/{cfg.chunk}/{cfg.bwd_chunk or cfg.chunk}"
    if rec.get("launch_shape") != shape:
        return None
    try:
        return int(int(rec["dram_bytes_per_launch"]) * n_inst / int(rec["instances"]))
    except (KeyError, ValueError, ZeroDivisionError):
        return None


def _time_refinement(rast, params, sc, dev, iters: int):
    """The refinement loop the rasterizer serves: `iters` Adam iterations of
    L1 RGB + 0.1 L1 depth against the keyframes' ray-cast targets over all
    views, through the differentiable render (Splat2DRender), every surfel
    parameter and every view's pose tangent optimised.  The surfels start
    from the workload with perturbed colours and opacities.  Times the loop
    (render, loss, backward, Adam step, clamps) with CUDA events after three
    untimed iterations; the loss is kept on the device every tenth iteration
    and read once at the end."""
    import torch

    from paper_2604_03092_gb300 import _abi
    from paper_2604_03092_gb300.rasterizer import render

    g = torch.Generator(device=dev).manual_seed(7)
    prm = [p.detach().clone() for p in params]
    prm[4] = (prm[4] + 0.1 * torch.randn(prm[4].shape, device=dev, generator=g)).clamp_(0.0, 1.0)
    prm[3] = prm[3] * (0.8 + 0.2 * torch.rand(prm[3].shape, device=dev, generator=g))
    prm = [p.requires_grad_(True) for p in prm]
    pose = torch.zeros(rast.n_views, 6, device=dev, requires_grad=True)
    opt = torch.optim.Adam([{"params": [prm[0]], "lr": 1e-4}, {"params": [prm[1]], "lr": 1e-5},
                            {"params": [prm[2]], "lr": 1e-3}, {"params": [prm[3]], "lr": 1e-2},
                            {"params": [prm[4]], "lr": 1e-2}])
    trgb = torch.from_numpy(sc.target_rgb).to(dev)
    tdep = torch.from_numpy(sc.target_depth).to(dev)
    rast.set_capacity(int(rast.capacity * 1.2))  # room for the instance count to grow as the surfels move
    losses = []

    def it(k):
        opt.zero_grad(set_to_none=False)
        rgb, depth, _, _ = render(rast, *prm, pose_tangent=pose, check=False)
        loss = (rgb - trgb).abs().mean() + 0.1 * (depth - tdep).abs().mean()
        loss.backward()
        opt.step()
        with torch.no_grad():
            prm[3].clamp_(0.01, 0.99)
            prm[1].clamp_(min=1e-6)
        if k % 10 == 0:
            losses.append(loss.detach())

    for k in range(3):
        it(-1)
    torch.cuda.synchronize()
    losses.clear()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for k in range(iters):
        it(k)
    b.record()
    torch.cuda.synchronize()
    status = rast.status()
    ms = a.elapsed_time(b) / iters
    return {"iterations": iters, "ms_per_iter": ms, "views_per_s": rast.n_views / (ms / 1e3),
            "loss_every_10": [float(x) for x in losses], "status": int(status),
            "status_ok": status == _abi.OK,
            "note": "Adam over means, scales, quats, opacity, rgb and every view's pose tangent; L1 RGB + 0.1 L1 "
                    "depth against the ray-cast keyframe targets; colours and opacities perturbed at the start"}


def _time_maintenance(rast, params, sc, out, dev, hbm_gbs, reps: int = 5):
    """CUDA-event times of the map-maintenance kernels on this workload:
    error attribution over all views (after a forward), the accumulation
    gate on one view's alpha, 2x2 voxelization of one keyframe-sized
    per-pixel map, and a per-keyframe Sim(3) correction of every surfel."""
    import torch

    from paper_2604_03092_gb300 import mapping
    from paper_2604_03092_gb300.rasterizer import accum_gate

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    res = {}
    rast.forward(*params, out=out, check=False)
    err = torch.rand(rast.n_pixels, device=dev)
    max_err = torch.zeros(rast.n_surfels, device=dev)
    res["max_error_ms"] = timed(lambda: rast.max_error(err, max_err))
    H, W = rast.sizes[0]
    alpha0 = out.alpha[:H * W]
    res["accum_gate_ms"] = timed(lambda: accum_gate(alpha0, 0.5))
    n = H * W
    g = torch.Generator(device=dev).manual_seed(0)
    m = torch.rand(n, 3, device=dev, generator=g) + torch.tensor([0.0, 0.0, 1.0], device=dev)
    q = torch.randn(n, 4, device=dev, generator=g)
    s_ = torch.rand(n, 2, device=dev, generator=g) * 0.01
    o = torch.rand(n, device=dev, generator=g)
    c = torch.rand(n, 3, device=dev, generator=g)
    vox_ms = timed(lambda: mapping.voxelize(m, q, s_, o, c, W, H, 0.05))
    res["voxelize_ms"] = vox_ms
    (_, _, _, _, _), _, n_out = mapping.voxelize(m, q, s_, o, c, W, H, 0.05)
    vox_bytes = 56 * n + 52 * int(n_out.item())  # attributes read (depths twice) + merged map written
    res["voxelize_hbm_frac"] = vox_bytes / (vox_ms / 1e3) / 1e9 / hbm_gbs
    N = rast.n_surfels
    mm, qq, ss = params[0].clone(), params[2].clone(), params[1].clone()
    kf = len(sc.views)
    sim3 = torch.cat([torch.randn(kf, 4, device=dev, generator=g), torch.randn(kf, 3, device=dev, generator=g) * 0.01,
                      torch.ones(kf, 1, device=dev)], 1).contiguous()
    index = (torch.arange(N, device=dev) * kf // N).to(torch.int32)
    sim_ms = timed(lambda: mapping.sim3_apply(mm, qq, ss, sim3, index))
    res["sim3_ms"] = sim_ms
    res["sim3_hbm_frac"] = (2 * 36 + 4) * N / (sim_ms / 1e3) / 1e9 / hbm_gbs
    res["note"] = (f"error attribution over {kf} views x {H}x{W}; gate on one {H}x{W} alpha map; voxelization of one "
                   f"{W}x{H} per-pixel map; Sim(3) of {N} surfels bound to {kf} keyframes")
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="submap32")
    ap.add_argument("--tile", default=None, help="WxH, e.g. 16x16 (default: autotune cache, else the shipped GB300 measurement, else 8x8)")
    ap.add_argument("--chunk", type=int, default=None)
    ap.add_argument("--fwd-tail", type=int, default=None, help="forward tail threshold per warp (255 = always)")
    ap.add_argument("--bwd-chunk", type=int, default=None, help="chunk of the backward pass (default: --chunk)")
    ap.add_argument("--autotune", action="store_true",
                    help="time every launch-shape candidate on this workload first (autotune.tune), then use the best")
    ap.add_argument("--plain-steps", type=int, default=2, help="steps of the per-view plain-launch baseline (0=skip)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--refine-iters", type=int, default=100,
                    help="Adam iterations of the refinement loop through Splat2DRender (0 = skip)")
    ap.add_argument("--cpu-views", type=int, default=4, help="whole views the oracle CPU baseline renders (~3 s each)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-maintenance", action="store_true", help="skip timing the map-maintenance kernels")
    ap.add_argument("--oracle-timing-child", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_timing_child:
        return oracle_timing_child()
    args.warmup = max(args.warmup, 3)

    wls = _workloads()
    if args.workload not in wls:
        raise SystemExit(f"unknown workload {args.workload}; choose from {sorted(wls)}")
    wl_desc, make = wls[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl_desc, make)

    import torch
    import torch.distributed as dist

    from paper_2604_03092_gb300 import autotune, multirank
    from paper_2604_03092_gb300.rasterizer import RasterConfig, Rasterizer

    ri = multirank.rank_info()
    world, rank, local = ri.world, ri.rank, ri.local
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    sc = make(multirank.submap_seed_offset(rank))  # each rank: its own independent submap
    V = len(sc.views)
    params = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in
              (sc.means, sc.scales, sc.quats, sc.opacity, sc.rgb)]

    cfg = RasterConfig(stats=True)
    tune_ms = None
    if args.autotune:
        gen = torch.Generator(device=dev).manual_seed(0)
        P = sum(v.width * v.height for v in sc.views)
        d_tune = (torch.randn(3 * P, device=dev, generator=gen) * 1e-6, torch.randn(P, device=dev, generator=gen) * 1e-7,
                  None, None)
        best, tune_ms = autotune.tune(sc.views, sc.n, autotune.cuda_runner(sc.views, params, d_tune), force=True)
        torch.cuda.empty_cache()
    tuned = autotune.lookup(sc.views, sc.n) if args.tile is None else None
    if tuned:
        cfg.tile_w, cfg.tile_h, cfg.chunk, cfg.bwd_chunk = tuned
    if args.tile:
        cfg.tile_w, cfg.tile_h = (int(x) for x in args.tile.lower().split("x"))
    if args.chunk:
        cfg.chunk = args.chunk
    if args.fwd_tail is not None:
        cfg.fwd_tail = args.fwd_tail
    if args.bwd_chunk is not None:
        cfg.bwd_chunk = args.bwd_chunk
    rast = Rasterizer(sc.views, sc.n, cfg, device=dev)
    im = rast.forward(*params)  # sizes the instance capacity (synchronises once)
    st0 = rast.stats()
    rast.set_capacity(int(st0["needed_capacity"] * 1.1) + 4096)

    # upstream gradient of L1 RGB + 0.1 L1 depth against the ray-cast targets
    if sc.target_rgb is not None and rast.uniform:
        shaped = rast.shaped(im)
        trgb = torch.from_numpy(sc.target_rgb).to(dev)
        tdep = torch.from_numpy(sc.target_depth).to(dev)
        d_rgb = (torch.sign(shaped.rgb - trgb) / trgb.numel()).contiguous().view(-1)
        d_depth = (0.1 * torch.sign(shaped.depth - tdep) / tdep.numel()).contiguous().view(-1)
    else:
        # no targets (views of different sizes): the same L1 RGB + 0.1 L1
        # depth gradient with random signs standing in for sign(render - target)
        gen = torch.Generator(device=dev).manual_seed(0)
        P = rast.n_pixels
        d_rgb = torch.sign(torch.randn(3 * P, device=dev, generator=gen)) / (3 * P)
        d_depth = 0.1 * torch.sign(torch.randn(P, device=dev, generator=gen)) / P
    d_out = (d_rgb, d_depth, None, None)
    out = rast.new_images()
    grads = rast.new_grads()
    stages = ["preprocess", "bin_sort", "render_fwd", "render_bwd", "preprocess_bwd"]

    def step(ev=None, prm=params, grd=grads):
        for t in grd:
            t.zero_()
        if ev is not None:
            ev[0].record()
        rast.preprocess(*prm)
        if ev is not None:
            ev[1].record()
        rast.bin_sort()
        if ev is not None:
            ev[2].record()
        rast.render_fwd(out)
        if ev is not None:
            ev[3].record()
        rast.render_bwd_tiles(d_out)
        if ev is not None:
            ev[4].record()
        rast.preprocess_bwd(*prm, grd)
        if ev is not None:
            ev[5].record()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if rast.status() != 0:
        raise SystemExit(f"device status {rast.status()} after warm-up")

    # ---- timed region: K steps, CUDA events around every stage -------------
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    launches0 = rast.launch_count()
    multirank.barrier()
    torch.cuda.synchronize()
    with ClockSampler(uuid) as clk:
        t_start.record()
        for k in range(args.steps):
            step(evs[k])
        t_end.record()
        torch.cuda.synchronize()
    launches = rast.launch_count() - launches0
    multirank.barrier()
    elapsed_ms = t_start.elapsed_time(t_end)
    stage_ms = {s: float(np.mean([evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(args.steps)]))
                for i, s in enumerate(stages)}
    st = rast.stats()
    if st["status"] != 0:
        raise SystemExit(f"device status {st['status']} in the timed region")
    max_ms = multirank.max_over_ranks(elapsed_ms, dev)
    views_all = multirank.sum_over_ranks(V * args.steps, dev)
    ms_per_step = max_ms / args.steps
    value = multirank.whole_job_rate(views_all, max_ms)

    # ---- the same step replayed from a CUDA graph ----------------------------
    graph_vps = None
    try:
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            step()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step()
        for _ in range(2):
            g.replay()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(args.steps):
            g.replay()
        b.record()
        torch.cuda.synchronize()
        graph_vps = V * args.steps / (a.elapsed_time(b) / 1e3)
        del g
    except Exception as e:  # report, do not hide
        graph_vps = f"failed: {e}"

    # ---- per-view plain launches (classic pattern: one view per launch
    #      sequence, a host sync per view to size the sort) -------------------
    plain_vps = None
    plain_stages = None
    if args.plain_steps > 0 and rank == 0:
        # one single-view rasterizer per distinct (image size, intrinsics,
        # surfel range), built before timing; each view re-uses its group's
        # rasterizer with its own pose
        groups = {}
        for v, vw in enumerate(sc.views):
            key = (vw.width, vw.height, float(vw.fx), float(vw.fy), float(vw.cx), float(vw.cy),
                   getattr(vw, "surfel_offset", 0), getattr(vw, "surfel_count", -1))
            groups.setdefault(key, []).append(v)
        singles = {}
        for key, vs in groups.items():
            one = Rasterizer([sc.views[vs[0]]], sc.n, cfg, device=dev)
            one_out = one.new_images()
            for v in vs:  # size the instance capacity for every view of the group
                for i, x in enumerate(sc.views[v].Rt.reshape(-1)):
                    one._cviews[0].Rt[i] = float(x)
                one.forward(*params, out=one_out, check=True)
            singles[key] = (one, one_out, one.new_grads())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nviews = 0
        for _ in range(args.plain_steps):
            for key, vs in groups.items():
                one, one_out, one_grads = singles[key]
                for v in vs:
                    for i, x in enumerate(sc.views[v].Rt.reshape(-1)):
                        one._cviews[0].Rt[i] = float(x)
                    o = int(rast._cviews[v].pixel_offset)
                    H, W = rast.sizes[v]
                    dv = (d_rgb[3 * o:3 * o + 3 * H * W], d_depth[o:o + H * W], None, None)
                    one.forward(*params, out=one_out, check=True)
                    one.render_bwd_tiles(dv)
                    one.preprocess_bwd(*params, one_grads)
                    nviews += 1
        torch.cuda.synchronize()
        plain_vps = nviews / (time.perf_counter() - t0)
        # where the per-view path spends its time: one more pass with CUDA
        # events around each of its stages (the status read is the host
        # synchronisation the per-view path needs to size its sort), and the
        # host wall time of the whole pass
        names = ["preprocess", "bin_sort", "render_fwd", "status_sync", "render_bwd", "preprocess_bwd"]
        acc = {n: 0.0 for n in names}
        t0 = time.perf_counter()
        nv = 0
        for key, vs in groups.items():
            one, one_out, one_grads = singles[key]
            for v in vs:
                one.set_view_pose(0, sc.views[v].Rt)
                o = int(rast._cviews[v].pixel_offset)
                H, W = rast.sizes[v]
                dv = (d_rgb[3 * o:3 * o + 3 * H * W], d_depth[o:o + H * W], None, None)
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
                ev[0].record()
                one.preprocess(*params)
                ev[1].record()
                one.bin_sort()
                ev[2].record()
                one.render_fwd(one_out)
                ev[3].record()
                if one.status() != 0:
                    raise SystemExit("device status in the per-view pass")
                ev[4].record()
                one.render_bwd_tiles(dv)
                ev[5].record()
                one.preprocess_bwd(*params, one_grads)
                ev[6].record()
                torch.cuda.synchronize()
                for i, n in enumerate(names):
                    acc[n] += ev[i].elapsed_time(ev[i + 1])
                nv += 1
        wall = (time.perf_counter() - t0) * 1e3 / nv
        plain_stages = {n: acc[n] / nv for n in names}
        plain_stages["host_wall_per_view"] = wall
        del singles

    # ---- end to end through the public API with host buffers -----------------
    # Every step copies its inputs (the surfel parameters) from pinned host
    # memory and reads its result (the parameter and pose gradients) back.
    # The copies run on a second stream and are double-buffered: step k+1's
    # parameters go up while step k computes, and step k's gradients come
    # down while step k+1 computes; events order each buffer's uses.
    pinned_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
                 (sc.means, sc.scales, sc.quats, sc.opacity, sc.rgb)]
    pinned_out = [[torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in grads] for _ in range(2)]
    h2d = sum(t.numel() * t.element_size() for t in pinned_in)
    d2h = sum(t.numel() * t.element_size() for t in pinned_out[0])
    prm_b = [params, [torch.empty_like(t) for t in params]]
    grd_b = [grads, rast.new_grads()]
    comp = torch.cuda.current_stream()
    copy_s = torch.cuda.Stream(device=dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]    # parameters of buffer b are on the device
    ev_comp = [torch.cuda.Event() for _ in range(2)]  # the step that used buffer b has finished
    ev_out = [torch.cuda.Event() for _ in range(2)]   # gradients of buffer b have reached the host
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(comp)
    copy_s.wait_stream(comp)
    with torch.cuda.stream(copy_s):
        for dst, src in zip(prm_b[0], pinned_in):
            dst.copy_(src, non_blocking=True)
        ev_in[0].record(copy_s)
    for k in range(args.e2e_steps):
        bi = k % 2
        comp.wait_event(ev_in[bi])
        if k >= 2:
            comp.wait_event(ev_out[bi])  # buffer bi's gradients from step k-2 have been read
        step(prm=prm_b[bi], grd=grd_b[bi])
        ev_comp[bi].record(comp)
        with torch.cuda.stream(copy_s):
            if k + 1 < args.e2e_steps:
                if k >= 1:
                    copy_s.wait_event(ev_comp[1 - bi])  # step k-1 no longer reads buffer 1-bi
                for dst, src in zip(prm_b[1 - bi], pinned_in):
                    dst.copy_(src, non_blocking=True)
                ev_in[1 - bi].record(copy_s)
            copy_s.wait_event(ev_comp[bi])
            for dst, src in zip(pinned_out[bi], grd_b[bi]):
                dst.copy_(src, non_blocking=True)
            ev_out[bi].record(copy_s)
    comp.wait_stream(copy_s)
    b.record(comp)
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b)
    e2e_vps = multirank.whole_job_rate(multirank.sum_over_ranks(V * args.e2e_steps, dev),
                                       multirank.max_over_ranks(e2e_ms, dev))
    del prm_b, grd_b

    # ---- the refinement loop (Sec. 4.3, "Lightweight Map Refinement") --------
    refine = None
    if args.refine_iters > 0 and rank == 0 and sc.target_rgb is not None and rast.uniform:
        refine = _time_refinement(rast, params, sc, dev, args.refine_iters)

    # ---- map maintenance around the refinement (Sec. 4.3), on this workload ---
    maint = None
    if not args.no_maintenance and rank == 0:
        maint = _time_maintenance(rast, params, sc, out, dev, _peaks()["hbm_gbs"])

    # ---- roofline of the dominant stage ------------------------------------------
    peaks = _peaks()
    clocks = clk.summary()
    lay = rast.layout
    n_vis = st["n_visible"]
    n_inst = st["n_instances"]
    # Each stage's ideal time is the largest of its algorithmic bytes over
    # the measured copy bandwidth, its FP32 lane-instructions over the FP32
    # lane rate and its special-function ops over the MUFU rate, with the
    # SM count read from the device and the maximum SM clock; the stage's
    # fraction is ideal / measured, and the binding term names its bound.
    n_sm = int(torch.cuda.get_device_properties(dev).multi_processor_count)
    clk_hz = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    instr_peak = n_sm * FP32_LANES_PER_SM * clk_hz      # lane-instructions / s
    mufu_peak = n_sm * MUFU_LANES_PER_SM * clk_hz
    bw = peaks["hbm_gbs"] * 1e9
    n_pix = rast.n_pixels
    pe_f, pe_b = st["fwd_pairs_evaluated"], st["bwd_pairs_evaluated"]
    work = {  # stage: (bytes, FP32 lane-instructions, MUFU ops)
        "preprocess": (56 * rast.n_surfels + 20 * lay.n_records + 80 * n_vis, 0, 0),
        "bin_sort": (32 * lay.n_records + 8 * n_inst + 20 * n_inst, 0, 0),
        "render_fwd": (FWD_BYTES_INST * n_inst + FWD_BYTES_PIX * n_pix, INSTR_FWD * pe_f, MUFU_FWD * pe_f),
        "render_bwd": (BWD_BYTES_INST * n_inst + BWD_BYTES_PIX * n_pix + BWD_BYTES_VIS * n_vis,
                       INSTR_BWD * pe_b, MUFU_BWD * pe_b),
        "preprocess_bwd": (4 * lay.n_records + 80 * n_vis + 56 * rast.n_surfels + 52 * rast.n_surfels, 0, 0),
    }
    stage_frac = {}
    t_ideal_sum = 0.0
    for s_ in stages:
        b_, i_, m_ = work[s_]
        t_ = stage_ms[s_] / 1e3
        terms = {"hbm": b_ / bw, "alu": i_ / instr_peak, "mufu": m_ / mufu_peak}
        bound = max(terms, key=terms.get)
        t_ideal_sum += terms[bound]
        stage_frac[s_] = {"bound": bound, "frac": terms[bound] / t_, "ms": stage_ms[s_],
                          "ideal_ms": terms[bound] * 1e3, "bytes": b_, "lane_instr": i_, "mufu": m_,
                          "achieved_gbs": b_ / t_ / 1e9, "frac_hbm": terms["hbm"] / t_,
                          "frac_alu": terms["alu"] / t_}
    stage_frac["render_fwd"]["flop"] = FLOP_EVAL * pe_f + FLOP_BLEND * st["fwd_pairs_blended"]
    stage_frac["render_bwd"]["flop"] = FLOP_EVAL * pe_b + FLOP_BWD * st["bwd_pairs_blended"]
    composite = t_ideal_sum / (sum(stage_ms.values()) / 1e3)
    dom = max(stage_ms, key=lambda s: stage_ms[s])
    sec = stage_ms[dom] / 1e3
    d = stage_frac[dom]
    traffic = _recorded_traffic(dom, cfg, n_inst)
    if d["bound"] == "hbm":
        roof = {"bound": "hbm", "kernel": dom, "achieved": d["bytes"] / sec / 1e9, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": d["frac"], "traffic": traffic,
                "peak_source": f"{peaks['source']} STREAM-style copy"}
    else:
        unit_peak = instr_peak if d["bound"] == "alu" else mufu_peak
        amount = d["lane_instr"] if d["bound"] == "alu" else d["mufu"]
        roof = {"bound": "alu", "kernel": dom, "achieved": amount / sec / 1e12, "peak": unit_peak / 1e12,
                "unit": "Tinstr/s", "frac": d["frac"], "traffic": traffic,
                "peak_source": (f"{n_sm} SMs (device) x {FP32_LANES_PER_SM if d['bound'] == 'alu' else MUFU_LANES_PER_SM}"
                                f" lanes x {clk_hz / 1e6:.0f} MHz")}
    roof["work"] = {"bytes": d["bytes"], "lane_instr": d["lane_instr"], "mufu": d["mufu"],
                    "frac_hbm": d["frac_hbm"], "frac_alu": d["frac_alu"], "sm_count": n_sm,
                    "per_unit": PER_UNIT.get(dom)}

    # ---- CPU baseline (the oracle, host cores, bounded sample) -----------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        per_view, desc, _ = oracle_views(sc, list(range(min(args.cpu_views, len(sc.views)))))
        cpu = {"value": 1.0 / per_view, "unit": "views/s", "cores": _omp_threads(), "kind": "oracle",
               "sample": desc, "breadth": oracle_timing()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "views/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "ms_per_view": ms_per_step / V,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded ray-cast indoor submap; stands in for ScanNet/BundleFusion)",
            "views_per_step": V, "config": _config(args, wl_desc, sc, world),
            "launch": {"tile": f"{cfg.tile_w}x{cfg.tile_h}", "chunk": cfg.chunk,
                       "bwd_chunk": cfg.bwd_chunk or cfg.chunk, "fwd_tail": cfg.fwd_tail, "instances": n_inst,
                       "visible_pairs": n_vis},
            "stages_ms": stage_ms, "stage_roofline": stage_frac, "composite_roofline_frac": composite,
            "roofline": roof, "clocks": clocks,
            "graph_views_per_s": graph_vps, "plain_per_view_views_per_s": plain_vps,
            "plain_per_view_stages_ms": plain_stages,
            "batched_stages_ms_per_view": {k: v / V for k, v in stage_ms.items()},
            "e2e": {"value": e2e_vps, "unit": "views/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "pairs": {k: st[k] for k in ("fwd_pairs_evaluated", "fwd_pairs_blended", "bwd_pairs_evaluated",
                                         "bwd_pairs_blended", "bwd_terms_outside")},
            "cpu_baseline": cpu,
            "refinement": refine,
            "autotune_ms": tune_ms,
            "map_maintenance": maint,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
