#!/usr/bin/env python
"""Throughput of the DRK splatting hot path on GB300: Mpix/s of one
forward + backward render (Sec. 4.4 pipeline and its reverse mode) of a
100k-primitive, K = 8, SH-degree-3 scene at 1920 x 1080, synthetic data.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl drk|reference]
    python bench.py --serve [--serve-requests R] [--serve-rate HZ] [--serve-batch B]
    python bench.py --order-study     (forward only: exact vs cache-sorting order)
    python bench.py --train           (training step with the fused Adam update)
    python bench.py --mesh            (mesh to DRK conversion and render)
    python bench.py --serve-sweep     (serving: max arrival rate within the latency target)

One process per GPU (torchrun for N > 1).  The path does not shard: every
rank renders its own replica of the workload ("replicas only"), value =
pixels of all ranks / max-over-ranks step time.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2412_11752_gb300 import synth  # noqa: E402

METRIC = "Mpix/s fwd+bwd at 1080p/100k DRK"
WORKLOAD = "clustered-100k-1080p"

# Algorithmic FP32 operations per (pixel, primitive) evaluation of Eq. 4 -
# Eq. 10 on the FMA/ALU pipes (one per add, mul, fma, compare, select; the
# atan2 polynomial counted as 16; transcendental MUFU ops not included).
OPS_PER_EVAL = 66
# extra operations per composited contributor in the backward (Eq. 1
# gradient, chain through Eq. 10 - Eq. 4 to the record quantities)
OPS_PER_EMIT_BWD = 190
# transcendental operations per evaluation: the reciprocal of the ray
# depth, the reciprocal inside the polar angle, the cosine of Eq. 6 and
# the exponentials of Eq. 8 and Eq. 10
XU_PER_EVAL = 5
# bytes the backward must read per composited contributor: its 32-byte
# record sector and its 4-byte grouped slot index
REC_BYTES_BWD = 36


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("drk", "reference"), default="drk")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-pixels", type=int, default=1024, help="oracle sample size (pixels, fwd+bwd)")
    ap.add_argument("--cull-level", type=int, default=2, choices=(0, 1, 2, 3),
                    help="tile culling: 0 none, 1 screen rectangle, 2 per-tile test (same image), "
                         "3 the paper's endpoint polygon (lossy)")
    ap.add_argument("--kbuf-capacity", type=int, default=16, choices=(8, 16, 32),
                    help="per-pixel depth-order buffer entries (any value gives the same image)")
    ap.add_argument("--serve", action="store_true",
                    help="serving mode: Poisson request mix through drk_serve (batched vs one at a time)")
    ap.add_argument("--serve-requests", type=int, default=160)
    ap.add_argument("--serve-rate", type=float, default=0.0, help="arrivals per second (0 = all at once)")
    ap.add_argument("--serve-batch", type=int, default=16)
    ap.add_argument("--serve-sweep", action="store_true",
                    help="serving headline: max arrival rate with p99 <= L* for batched and one-at-a-time serving")
    ap.add_argument("--train", action="store_true",
                    help="training step: render + L1 gradient + backward + fused Adam (activations included)")
    ap.add_argument("--mesh", action="store_true",
                    help="mesh to DRK: conversion of a 518k-triangle wall and its 1080p render with depth and normal")
    ap.add_argument("--order-study", action="store_true",
                    help="forward-only comparison of the exact order with the paper's cache-sorting order")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


RASTER_SOURCES = ("paper_2412_11752_gb300/csrc/raster.cu", "paper_2412_11752_gb300/csrc/drk_common.cuh",
                  "paper_2412_11752_gb300/csrc/drk_internal.h")


def raster_traffic(workload: str):
    """DRAM bytes of one forward raster launch from the committed ncu summary
    of this workload, or None if there is none or the raster sources changed
    since it was captured (the summary records their hash)."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", f"raster_fwd_dram_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"source hash \| `([0-9a-f]+)`", text)
    t = re.search(r"traffic per launch \| ([0-9.]+) GB", text)
    if not m or not t:
        return None
    h = hashlib.sha256()
    for f in RASTER_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return float(t.group(1)) * 1e9 if h.hexdigest()[:16] == m.group(1) else None


def records_roofline(n_records: int, ms: float, fma_ops: float, xu_s_per_unit: float, hbm_gbs: float,
                     replayed: bool = False, hbm_basis: str = ""):
    """The backward over the contributor records, reported like the forward
    raster: per record the pair is evaluated again (OPS_PER_EVAL FP32 and
    XU_PER_EVAL transcendental operations) and its gradient chained
    (OPS_PER_EMIT_BWD more), against the measured FMA rate (fma_ops, per
    second) and transcendental mix (xu_s_per_unit seconds per evaluation's
    XU_PER_EVAL operations); and its REC_BYTES_BWD algorithmic bytes per
    record against the measured copy rate.  n_records counts every
    composited contributor, which includes those of tiles taken by the
    exact replay when `replayed`.  None without records or time."""
    if n_records <= 0 or ms <= 0.0 or fma_ops <= 0.0 or xu_s_per_unit <= 0.0 or hbm_gbs <= 0.0:
        return None
    s = ms / 1e3
    ops = OPS_PER_EVAL + OPS_PER_EMIT_BWD
    fma_peak = fma_ops / 1e12
    achieved = n_records * ops / s / 1e12
    xu_peak = XU_PER_EVAL / xu_s_per_unit / 1e12
    xu_achieved = n_records * XU_PER_EVAL / s / 1e12
    gbs = n_records * REC_BYTES_BWD / s / 1e9
    return {"kernel": "raster_bwd_records", "bound": "alu", "achieved": achieved, "peak": fma_peak, "unit": "Top/s",
            "frac": achieved / fma_peak, "ops_per_unit": ops, "units": int(n_records), "ms": ms,
            "replayed_tiles": bool(replayed),
            "xu": {"achieved": xu_achieved, "peak": xu_peak, "unit": "Top/s", "frac": xu_achieved / xu_peak,
                   "ops_per_unit": XU_PER_EVAL},
            "hbm": {"bytes_per_unit": REC_BYTES_BWD, "achieved_gbs": gbs, "peak_gbs": hbm_gbs, "frac": gbs / hbm_gbs,
                    "peak_basis": hbm_basis}}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


def hbm_peak() -> tuple[float, str]:
    """The HBM denominator and its basis: the copy rate measured on this
    pool's GPUs when MEASURED_PEAKS.json holds it, else an earlier GB300
    measurement of 6.8 TB/s."""
    v = measured_peaks().get("hbm_gbs")
    if v:
        return float(v), "hbm_gbs of MEASURED_PEAKS.json (of measured)"
    return 6800.0, "6800 GB/s from an earlier GB300 measurement (of fallback)"


def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_step: float, ms_step_local: float, world: int, device) -> tuple[float, float]:
    """Whole-job rate of `world` independent replicas: the units of all ranks
    divided by the slowest rank's step time (ms), and that step time."""
    ms = max_over_ranks(ms_step_local, world, device)
    return world * units_per_step / (ms / 1e3), ms


# ---------------------------------------------------------------------------
def oracle_rate(scene, cam, pixels: int, seed: int = 7) -> tuple[float, dict]:
    """Oracle (FP64 CPU) forward + backward over a seeded pixel sample: Mpix/s."""
    from oracle import drk_oracle as O
    opt = O.Options(alpha_min=float(np.float32(np.exp(-9.0))), T_min=float(np.float32(1e-4)),
                    alpha_max=float(np.float32(0.99)), lowpass_sl=float(np.float32(0.70710678)),
                    near=float(np.float32(0.2)))
    pix = synth.pixel_sample(cam.width, cam.height, pixels, seed=seed)
    g = np.random.default_rng(seed).standard_normal((pix.shape[0], 3))
    t0 = time.perf_counter()
    O.render_pixels(scene, cam, opt, pix)
    O.render_backward_pixels(scene, cam, opt, pix, g)
    dt = time.perf_counter() - t0
    info = {"cores": O.max_threads(),
            "sample": f"{pix.shape[0]} seeded pixels of the {cam.width}x{cam.height} frame, forward + backward "
                      f"(brute force over all {scene.n} primitives per pixel, FP64)",
            "seconds": dt}
    return pix.shape[0] / dt / 1e6, info


def run_reference(args):
    rank, world, local = dist_setup()
    if rank != 0:
        return 0
    sc_f, cam_f = synth.WORKLOADS[args.workload]
    scene, cam = sc_f(), cam_f()
    px = max(16, args.cpu_pixels // 4)
    for _ in range(max(0, args.warmup)):
        oracle_rate(scene, cam, 16, seed=1)
    rates, infos = [], []
    t0 = time.perf_counter()
    for k in range(args.steps):
        r, info = oracle_rate(scene, cam, px, seed=100 + k)
        rates.append(r)
        infos.append(info)
    wall = time.perf_counter() - t0
    value = args.steps * px / sum(i["seconds"] for i in infos) / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "pixels_per_step": px, "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": infos[0]["cores"], "kind": "oracle",
                             "sample": infos[0]["sample"].replace(f"{px} seeded", f"{px} seeded (per step)")},
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
def run_drk(args):
    import torch
    rank, world, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2412_11752_gb300 import drk

    sc_f, cam_f = synth.WORKLOADS[args.workload]
    scene, cam = sc_f(), cam_f()
    H, W = cam.height, cam.width
    ds = drk.DeviceScene.from_scene(scene, dev)
    target = torch.from_numpy(synth.target_image(H, W)).to(dev)
    opt = drk.Options(kbuf_capacity=args.kbuf_capacity, cull_level=args.cull_level)
    ctx = drk.Context(local)
    out = dict(rgb=torch.empty((3, H, W), device=dev), T=None, n=None)
    inv_n = 1.0 / float(3 * H * W)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def step(scene_dev):
        rgb, _, _, st = drk.drk_render(scene_dev, cam, opt, ctx=ctx, need_state=True, out=out)
        dL = torch.sign(rgb - target).mul_(inv_n)      # d(mean |C - target|)/dC
        g = drk.drk_render_backward(scene_dev, cam, opt, st, dL, ctx=ctx)
        st.free()
        return rgb, g

    for _ in range(max(1, args.warmup)):
        step(ds)
    torch.cuda.synchronize()
    # The raster's statistics (evaluations, contributors, heap spills) are
    # the same for every render of this frame: they are taken from the last
    # warm-up step, and the timed and end-to-end steps run the forward
    # without them, as a user who does not read them would
    stats = ctx.stats()
    ctx.stats_enable(False)

    # ---- device-timed region
    props = torch.cuda.get_device_properties(dev)
    gpu_id = getattr(props, "uuid", None)
    gpu_id = f"GPU-{gpu_id}" if gpu_id is not None and not str(gpu_id).startswith("GPU-") else (gpu_id or str(local))
    sampler = ClockSampler(str(gpu_id))
    ctx.timing_enable(True)
    l0 = drk.launch_count()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()                                  # evict L2 between steps (untimed)
        starts[k].record()
        step(ds)
        ends[k].record()
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    launches = drk.launch_count() - l0
    stage = ctx.timing_read()
    ctx.timing_enable(False)
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # median step (robust to the odd slow step); spread reported beside it
    value, ms_step = replica_rate(H * W / 1e6, float(np.median(ms)), world, dev)
    spread = {"min": float(np.min(ms)), "p10": float(np.percentile(ms, 10)), "median": float(np.median(ms)),
              "p90": float(np.percentile(ms, 90)), "max": float(np.max(ms)), "mean": float(np.mean(ms))}

    # ---- roofline of the dominant kernel: FP32 FMA pipe and transcendental
    # unit, both measured on this GPU by the library's own kernels
    pipes = drk.measure_pipes(local)
    peaks = measured_peaks()
    sms = props.multi_processor_count
    smax = float(peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0)
    fma_peak = pipes["fma_ops"] / 1e12
    fwd_ms = stage["raster"][0] / max(1, stage["raster"][1])
    bwd_ms = stage["raster_bwd"][0] / max(1, stage["raster_bwd"][1])
    if fwd_ms >= bwd_ms:
        dom, dom_ms, units = "raster_fwd", fwd_ms, stats["n_evals"]
        ops_unit, xu_unit = OPS_PER_EVAL, XU_PER_EVAL
    else:
        # the records kernel re-evaluates each composited pair and chains its gradient
        dom, dom_ms, units = "raster_bwd", bwd_ms, stats["n_emitted"]
        ops_unit, xu_unit = OPS_PER_EVAL + OPS_PER_EMIT_BWD, XU_PER_EVAL
    achieved = units * ops_unit / (dom_ms / 1e3) / 1e12
    # seconds per transcendental op of the evaluation's mix (2 ex2, 2 rcp, 1 cos)
    xu_s_per_unit = 2.0 / pipes["ex2_ops"] + 2.0 / pipes["rcp_ops"] + 1.0 / pipes["cos_ops"]
    xu_peak = xu_unit / xu_s_per_unit / 1e12
    xu_achieved = units * xu_unit / (dom_ms / 1e3) / 1e12
    roof_ms = 1e3 * max(units * ops_unit / pipes["fma_ops"], units * xu_s_per_unit)
    sm_load = float(clocks.get("sm_mhz") or smax)
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fma_peak, "unit": "Top/s",
                "frac": achieved / fma_peak, "traffic": raster_traffic(args.workload) if dom == "raster_fwd" else None,
                "peak_basis": "FP32 FMA ops/s measured by drk_measure_pipes on this GPU (of measured)",
                "ops_per_unit": ops_unit, "units": units,
                "units_basis": "counters of the last warm-up step (timed steps run the raster without statistics)",
                "xu": {"achieved": xu_achieved, "peak": xu_peak, "unit": "Top/s", "frac": xu_achieved / xu_peak,
                       "ops_per_unit": xu_unit, "peak_basis": "2 ex2 + 2 rcp + 1 cos at the measured MUFU rates"},
                "roofline_time_ms": roof_ms, "roofline_frac": roof_ms / dom_ms,
                "nominal_fma_peak": sms * 128 * smax * 1e6 / 1e12,
                "measured_pipes_tops": {k: v / 1e12 for k, v in pipes.items() if k.endswith("_ops")},
                "load_clock_mhz": sm_load}
    # HBM-bound stages: algorithmic bytes per launch over their event times
    hbm, hbm_basis = hbm_peak()
    P, N, K = stats["n_pairs"], scene.n, scene.K
    rec_b = 4 * (24 + 4 * (8 if K <= 8 else 16))
    bnd_b = 4 * (((10 + (8 if K <= 8 else 16) + 3) + 3) // 4 * 4)
    par_b = 4 * (3 + 4 + 2 * K + 3 + 3 * (scene.sh_degree + 1) ** 2)
    stage_bytes = {
        # 4 passes of 8-bit digits: keys and values read and written; tile ranges read the keys
        "sort": 4 * P * 16 + 4 * P,
        # parameters read; raster record, culling bound and colour written; the
        # culling count reads record and bound and writes a count; scan of the counts
        "preprocess": N * (par_b + rec_b + bnd_b + 12) + N * (rec_b + bnd_b + 4) + N * 12,
        # record and bound read per primitive; (key, value) written per pair
        "emit": N * (rec_b + bnd_b) + P * 8,
    }
    hbm_stages = {}
    for k, b in stage_bytes.items():
        if stage.get(k, (0, 0))[1]:
            ms_k = stage[k][0] / stage[k][1]
            gbs = b / (ms_k / 1e3) / 1e9
            hbm_stages[k] = {"bytes": b, "ms": ms_k, "achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm,
                             "peak_basis": hbm_basis}
    # the backward's records kernel beside the dominant kernel
    bwd_roof = records_roofline(stats["n_emitted"], bwd_ms, pipes["fma_ops"], xu_s_per_unit, hbm,
                                stats["n_replay_evals"] > 0, hbm_basis)
    if bwd_roof is not None:
        roofline["backward"] = bwd_roof

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        host_params = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k), np.float32)).pin_memory()
                       for k in drk.PARAM_NAMES}
        host_rgb = torch.empty((3, H, W), dtype=torch.float32).pin_memory()
        host_grads = {k: torch.empty_like(v).pin_memory() for k, v in host_params.items()}
        dev_params = {k: torch.empty(v.shape, dtype=torch.float32, device=dev) for k, v in host_params.items()}
        h2d = sum(v.numel() * 4 for v in host_params.values())
        d2h = host_rgb.numel() * 4 + sum(v.numel() * 4 for v in host_grads.values())
        e_steps = max(3, args.steps // 2)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            for k in drk.PARAM_NAMES:
                dev_params[k].copy_(host_params[k], non_blocking=True)
            sd = drk.DeviceScene(**dev_params, sh_degree=scene.sh_degree)
            rgb, g = step(sd)
            host_rgb.copy_(rgb, non_blocking=True)
            for k in drk.PARAM_NAMES:
                host_grads[k].copy_(g[k], non_blocking=True)
            torch.cuda.synchronize()
        wall = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": world * e_steps * H * W / wall / 1e6, "unit": "Mpix/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
    ctx.stats_enable(True)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, info = oracle_rate(scene, cam, args.cpu_pixels)
        cpu = {"value": r, "unit": "Mpix/s", "cores": info["cores"], "kind": "oracle", "sample": info["sample"]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "primitives": scene.n, "K": scene.K,
                           "sh_degree": scene.sh_degree, "width": W, "height": H, "tile": 16,
                           "cull_level": opt.cull_level, "kbuf_capacity": opt.kbuf_capacity,
                           "step": "render + L1-loss gradient + backward to all parameters",
                           "l2": "flushed between timed steps (256 MiB write)",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roofline, "hbm_stages": hbm_stages, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches,
                "clocks": clocks, "step_ms_spread": spread, "statistic": "median step time",
                "stages_ms": {k: v[0] / max(1, v[1]) for k, v in stage.items() if v[1]},
                "counters": {k: stats[k] for k in ("n_pairs", "n_evals", "n_geo_evals", "n_contrib_evals", "n_emitted",
                                                   "n_spills", "n_replay_evals",
                                                   "n_extra_passes", "n_visible")}}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def order_study(args):
    """Forward-only render time and image of the exact (r_t, index) order
    against the cache-sorting order (Sec. 4.4, centre-depth pre-sort, a
    cache of 8 or 16 entries), on the bench workload.  One JSON line."""
    import torch
    from paper_2412_11752_gb300 import drk
    dev = torch.device("cuda", 0)
    sc_f, cam_f = synth.WORKLOADS[args.workload]
    scene, cam = sc_f(), cam_f()
    H, W = cam.height, cam.width
    ds = drk.DeviceScene.from_scene(scene, dev)
    ctx = drk.Context(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    modes = {"exact": drk.Options(), "cache8": drk.Options(order_mode=1, kbuf_capacity=8),
             "cache16": drk.Options(order_mode=1, kbuf_capacity=16),
             # the paper's tile culling as printed (Eq. 11 - Eq. 12), alone and
             # with the cache: the whole pipeline as the paper states it
             "exact_papercull": drk.Options(cull_level=drk.CULL_PAPER),
             "cache8_papercull": drk.Options(order_mode=1, kbuf_capacity=8, cull_level=drk.CULL_PAPER)}
    res, imgs = {}, {}
    for name, opt in modes.items():
        out = dict(rgb=torch.empty((3, H, W), device=dev), T=None, n=None)
        for _ in range(args.warmup):
            drk.drk_render(ds, cam, opt, ctx=ctx, out=out)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        ctx.timing_enable(True)
        for a, b in ev:
            flush.zero_()
            a.record()
            drk.drk_render(ds, cam, opt, ctx=ctx, out=out)
            b.record()
        torch.cuda.synchronize()
        stage = ctx.timing_read()
        ctx.timing_enable(False)
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        imgs[name] = out["rgb"].clone()
        res[name] = {"ms_per_frame": ms, "mpix_s": H * W / ms / 1e3, "pairs": ctx.stats()["n_pairs"],
                     "stages_ms": {k: v[0] / max(1, v[1]) for k, v in stage.items() if v[1]}}
    for name in [m for m in modes if m != "exact"]:
        d = (imgs[name] - imgs["exact"]).abs()
        mse = float(((imgs[name] - imgs["exact"]) ** 2).mean())
        res[name]["vs_exact"] = {"max_abs": float(d.max()), "mean_abs": float(d.mean()),
                                 "psnr_db": 10 * np.log10(1.0 / mse) if mse > 0 else None,
                                 "pixels_over_1e-3": int((d.amax(0) > 1e-3).sum())}
        res[name]["speedup_vs_exact"] = res["exact"]["ms_per_frame"] / res[name]["ms_per_frame"]
    print(json.dumps({"metric": "Mpix/s forward, exact vs cache-sorting order", "unit": "Mpix/s",
                      "steps": args.steps, "warmup": args.warmup, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": args.workload, "primitives": scene.n, "width": W, "height": H,
                                 "l2": "flushed between timed frames (256 MiB write)"},
                      "modes": res}), flush=True)
    return 0


def train_bench(args):
    """Training steps of 100k DRKs (K = 8, SH degree 3) fitted to a synthetic
    1920 x 1080 shape image: render with a backward state, L1 gradient,
    render backward, fused activation backward + Adam + activation
    (supplementary "Parametrization" and "Model Training").  One JSON line
    with the step rate and the Adam kernel against the HBM roofline."""
    import torch
    from paper_2412_11752_gb300 import drk
    dev = torch.device("cuda", 0)
    n, K, sh, W, H = 100_000, 8, 3, 1920, 1080
    cam = synth.camera_front(W, H)
    raw = drk.RawScene.from_arrays(synth.raw_scene(n, K, seed=6002, sh_degree=sh), sh_degree=sh, device=dev)
    target = torch.from_numpy(synth.shape_target(H, W)).to(dev)
    opt = drk.Adam(raw)
    ropt = drk.Options(bg=(0.35, 0.35, 0.35))
    ctx = drk.Context(0)
    out = dict(rgb=torch.empty((3, H, W), device=dev), T=None, n=None)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    inv_n = 1.0 / float(3 * H * W)
    losses = []

    def step(k, ev=None):
        rgb, _, _, st = drk.drk_render(opt.scene, cam, ropt, ctx=ctx, need_state=True, out=out)
        diff = rgb - target
        losses.append(diff.abs().mean())
        g = drk.drk_render_backward(opt.scene, cam, ropt, st, torch.sign(diff).mul_(inv_n), ctx=ctx)
        st.free()
        if ev is not None:
            ev[0].record()
        opt.step(g, drk.learning_rates(k, 35000))
        if ev is not None:
            ev[1].record()

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    mk = lambda: torch.cuda.Event(enable_timing=True)
    st_ev = [(mk(), mk()) for _ in range(args.steps)]
    ad_ev = [(mk(), mk()) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        st_ev[k][0].record()
        step(args.warmup + k, ad_ev[k])
        st_ev[k][1].record()
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in st_ev]))
    adam_ms = float(np.mean([a.elapsed_time(b) for a, b in ad_ev]))
    ncol = 3 * (sh + 1) ** 2
    # algorithmic bytes of one update: every raw float read with its gradient
    # and two moments, written back with the moments (28 B); activated
    # arrays written once more (quat, K scales, K angles, eta, tau, opacity)
    floats = 3 + 4 + 2 * K + 3 + ncol
    adam_bytes = n * (28 * floats + 4 * (7 + 2 * K))
    peak, peak_basis = hbm_peak()
    achieved = adam_bytes / (adam_ms / 1e3) / 1e9
    print(json.dumps({"metric": "training steps/s (render + backward + fused Adam) at 1080p/100k DRK",
                      "value": 1e3 / ms, "unit": "steps/s", "ms_per_step": ms, "mpix_s": H * W / ms / 1e3,
                      "steps": args.steps, "warmup": args.warmup, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "train-100k-1080p (raw init, shape target)", "primitives": n, "K": K,
                                 "sh_degree": sh, "width": W, "height": H,
                                 "l2": "flushed between timed steps (256 MiB write)"},
                      "adam": {"ms": adam_ms, "bytes_per_launch": adam_bytes,
                               "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                            "frac": achieved / peak, "peak_basis": peak_basis}},
                      "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
                      "gpu_launches_adam_per_step": 1}), flush=True)
    return 0


def mesh_bench(args):
    """Mesh to DRK (Sec. 5.4): conversion of a 720 x 360-cell triangulated
    height-field wall (518,400 faces, K = 3) and its 1920 x 1080 render:
    exact order, exact with depth and normal images, and the cache-sorting
    order (the supplement notes that converted meshes depend on the order;
    that mode packs a centre-depth rank into the 19 depth bits of a 1080p
    pair key, so it takes at most 2^19 primitives).  One JSON line."""
    import torch
    from paper_2412_11752_gb300 import drk
    dev = torch.device("cuda", 0)
    W, H = 1920, 1080
    verts, faces = synth.mesh_heightfield(720, 360, seed=7003, triangles=True)
    colors = synth.mesh_colors(len(faces), seed=7203)
    v, f, c = (torch.from_numpy(x).to(dev) for x in (verts, faces, colors))
    mopt = drk.MeshOptions(K=3, tau=0.95)
    cam = synth.camera_front(W, H)
    ctx = drk.Context(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    mk = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev = [(mk(), mk()) for _ in range(args.steps)]
        for a, b in ev:
            flush.zero_()
            a.record()
            fn()
            b.record()
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    holder = {}

    def convert():
        holder["sc"], holder["st"] = drk.mesh_to_drk(v, f, c, mopt)

    conv_ms = timed(convert)
    sc, st = holder["sc"], holder["st"]
    n_rejected = int((st != 0).sum())
    nf = len(faces)
    # algorithmic bytes per face: the index row and three gathered vertices
    # and the colour read; mu, quat, scale, theta, eta, tau, opacity, colour
    # and status written
    bytes_face = 4 * 3 + 3 * 12 + 12 + 4 * (3 + 4 + 3 + 3 + 1 + 1 + 1 + 3) + 4
    peak, peak_basis = hbm_peak()
    res = {}
    imgs = {}
    for name, opt, aux in (("exact", drk.Options(), False), ("exact_depth_normal", drk.Options(), True),
                           ("cache8", drk.Options(order_mode=1, kbuf_capacity=8), False)):
        out = dict(rgb=torch.empty((3, H, W), device=dev), T=torch.empty((H, W), device=dev), n=None)
        if aux:
            out["depth"] = torch.empty((H, W), device=dev)
            out["normal"] = torch.empty((3, H, W), device=dev)
        ctx.timing_enable(True)
        ms = timed(lambda: drk.drk_render(sc, cam, opt, ctx=ctx, out=out))
        stage = ctx.timing_read()
        ctx.timing_enable(False)
        imgs[name] = out["rgb"].clone()
        res[name] = {"ms_per_frame": ms, "mpix_s": H * W / ms / 1e3,
                     "stages_ms": {k: v_[0] / max(1, v_[1]) for k, v_ in stage.items() if v_[1]}}
        if aux:
            cov = (1.0 - out["T"]).clamp_min(1e-6)
            inner = cov > 0.9
            res[name]["mean_depth_covered"] = float((out["depth"] / cov)[inner].mean())
    d = (imgs["cache8"] - imgs["exact"]).abs()
    mse = float(((imgs["cache8"] - imgs["exact"]) ** 2).mean())
    res["cache8"]["vs_exact"] = {"max_abs": float(d.max()), "mean_abs": float(d.mean()),
                                 "psnr_db": 10 * np.log10(1.0 / mse) if mse > 0 else None,
                                 "pixels_over_1e-3": int((d.amax(0) > 1e-3).sum())}
    print(json.dumps({"metric": "mesh to DRK: faces/s converted and 1080p frames/s rendered", "unit": "faces/s",
                      "value": nf / (conv_ms / 1e3), "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
                      "data": "synthetic", "config": {"workload": "heightfield-518k-tri-1080p", "faces": nf, "K": 3,
                                                      "tau": 0.95, "width": W, "height": H,
                                                      "l2": "flushed between timed calls (256 MiB write)"},
                      "convert": {"ms": conv_ms, "rejected": n_rejected,
                                  "roofline": {"bound": "hbm", "achieved": nf * bytes_face / (conv_ms / 1e3) / 1e9,
                                               "peak": peak, "unit": "GB/s",
                                               "frac": nf * bytes_face / (conv_ms / 1e3) / 1e9 / peak,
                                               "peak_basis": peak_basis, "bytes_per_face": bytes_face}},
                      "render": res}), flush=True)
    return 0


def serve_run(D, torch, dscenes, reqs, max_batch: int, budget: int) -> dict:
    """Replays (arrival_s, scene, camera) requests through one server; latency
    = completion - arrival of each request, throughput over the whole run."""
    outs = [torch.empty((3, c.height, c.width), device="cuda") for _, _, c in reqs]
    torch.cuda.synchronize()
    with D.Server(0, mem_budget=budget, max_batch=max_batch) as srv:
        ids = [srv.add_scene(d) for d in dscenes]
        # warm-up: four requests fill the server's memory pool
        for _, sid, cam in reqs[:4]:
            o = torch.empty((3, cam.height, cam.width), device="cuda")
            srv.release(_wait_release(srv, srv.submit(ids[sid], cam, o)))
        t0 = time.perf_counter()
        tickets = []
        for (arr, sid, cam), o in zip(reqs, outs):
            dt = arr - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(ids[sid], cam, o))
        tm = [srv.wait(t, 600000) for t in tickets]
        tl = [srv.timeline(t, 600000) for t in tickets]
    bad = [t["status"] for t in tm if t["status"] != 0]
    overlap = batch_overlap(tl)
    lat = np.array([t["end_ms"] - t["arrival_ms"] for t in tm])
    span_ms = max(t["end_ms"] for t in tm) - min(t["arrival_ms"] for t in tm)
    px = sum(c.width * c.height for _, _, c in reqs)
    return {"max_batch": max_batch, "frames_per_s": len(reqs) / (span_ms / 1e3), "Mpix_per_s": px / (span_ms / 1e3) / 1e6,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_batch": float(np.mean([t["batch_size"] for t in tm])), "failed": len(bad), "overlap": overlap}


def batch_overlap(timelines) -> dict:
    """Device-timeline evidence of overlap between batches: for every batch,
    the share of its phases A and B (preprocess, culling, emission, sort)
    that ran while a batch on the other stream was rasterising, and how
    much of the total device time two batches were active at once."""
    batches = {}
    for t in timelines:
        if t["status"] == 0 and t["dev_r1_ms"] > 0:
            batches[(t["stream"], t["dev_a0_ms"])] = (t["dev_a0_ms"], t["dev_b1_ms"], t["dev_r1_ms"], t["stream"])
    bl = sorted(batches.values())
    if not bl:
        return {}
    ab_total = ab_over = 0.0
    for a0, b1, r1, s in bl:
        ab_total += b1 - a0
        for a0o, b1o, r1o, so in bl:
            if so != s:
                ab_over += max(0.0, min(b1, r1o) - max(a0, b1o))
    # time with two batches active (any phase) against the span
    ev = sorted([(a0, 1) for a0, _, _, _ in bl] + [(r1, -1) for _, _, r1, _ in bl])
    both = busy = 0.0
    act, last = 0, ev[0][0]
    for x, d in ev:
        if act >= 1:
            busy += x - last
        if act >= 2:
            both += x - last
        act += d
        last = x
    return {"batches": len(bl), "phase_ab_ms": ab_total, "phase_ab_under_other_raster_ms": ab_over,
            "phase_ab_overlap_frac": ab_over / ab_total if ab_total > 0 else 0.0,
            "device_busy_ms": busy, "two_batches_active_ms": both,
            "mean_raster_ms": float(np.mean([r1 - b1 for _, b1, r1, _ in bl])),
            "mean_phase_ab_ms": ab_total / len(bl)}


def _wait_release(srv, tk):
    srv.wait(tk, 600000)
    return tk


def run_serve(args):
    import torch
    from paper_2412_11752_gb300 import drk as D
    D.lib()
    scenes = synth.serve_scenes()
    dscenes = [D.DeviceScene.from_scene(s, "cuda") for s in scenes]
    reqs = synth.serve_requests(args.serve_requests, len(scenes), args.serve_rate)
    budget = 64 << 30
    res = {"metric": "serving throughput and latency, Poisson request mix", "impl": "drk-serve",
           "data": "synthetic", "requests": len(reqs), "rate_hz": args.serve_rate,
           "config": {"scenes": [s.n for s in scenes], "resolutions": list(synth.SERVE_RESOLUTIONS),
                      "weights": list(synth.SERVE_RES_WEIGHTS), "mem_budget": budget}}
    res["batched"] = serve_run(D, torch, dscenes, reqs, args.serve_batch, budget)
    res["one_at_a_time"] = serve_run(D, torch, dscenes, reqs, 1, budget)
    print(json.dumps(res), flush=True)
    return 0


def serve_sequential(D, torch, dscenes, reqs) -> dict:
    """One request at a time without a server: each request, in arrival
    order, is rendered with drk_render once it has arrived and the host waits
    for it before taking the next; latency = completion - arrival."""
    ctx = D.Context(0)
    outs = [dict(rgb=torch.empty((3, c.height, c.width), device="cuda"), T=None, n=None) for _, _, c in reqs]
    for _, sid, cam in reqs[:4]:                       # warm-up, as for the server
        D.drk_render(dscenes[sid], cam, ctx=ctx, out=dict(rgb=torch.empty((3, cam.height, cam.width), device="cuda"),
                                                          T=None, n=None))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat, ends = [], []
    for (arr, sid, cam), o in zip(reqs, outs):
        dt = arr - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        D.drk_render(dscenes[sid], cam, ctx=ctx, out=o)
        torch.cuda.synchronize()
        now = time.perf_counter() - t0
        lat.append((now - arr) * 1e3)
        ends.append(now)
    span = max(ends) - min(a for a, _, _ in reqs)
    px = sum(c.width * c.height for _, _, c in reqs)
    return {"max_batch": 1, "frames_per_s": len(reqs) / span, "Mpix_per_s": px / span / 1e6,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)), "mean_batch": 1.0,
            "failed": 0}


def serve_sweep(args):
    """Serving headline: L* = p99 latency of one-at-a-time serving at half of
    its saturation rate; for each mode, the largest Poisson arrival rate of
    a grid whose p99 stays within L*.  One JSON line."""
    import torch
    from paper_2412_11752_gb300 import drk as D
    D.lib()
    scenes = synth.serve_scenes()
    dscenes = [D.DeviceScene.from_scene(s, "cuda") for s in scenes]
    budget = 64 << 30
    nreq = args.serve_requests
    # "sequential": drk_render one request at a time (no server);
    # "server_batch1": the server with batches of one (consecutive requests
    # still overlap on its two streams); "batched": batches of up to max_batch
    modes = {"batched": args.serve_batch, "server_batch1": 1, "sequential": 0}

    def run(m, lam):
        reqs = synth.serve_requests(nreq, len(scenes), lam)
        if modes[m] == 0:
            return serve_sequential(D, torch, dscenes, reqs)
        return serve_run(D, torch, dscenes, reqs, modes[m], budget)

    sat = {m: run(m, 0.0) for m in modes}
    x1 = sat["sequential"]["frames_per_s"]
    L = run("sequential", 0.5 * x1)["p99_ms"]
    grid = [round(f * x1, 2) for f in (0.4, 0.5, 0.6, 0.8, 1.0, 1.2)]
    runs, best = {m: [] for m in modes}, {}
    for m in modes:
        best[m] = None
        for lam in grid:
            r = run(m, lam)
            runs[m].append({"rate_hz": lam, "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"],
                            "frames_per_s": r["frames_per_s"], "mean_batch": r["mean_batch"],
                            "overlap": r.get("overlap")})
            if r["p99_ms"] <= L:
                best[m] = lam
    print(json.dumps({"metric": "max Poisson arrival rate with p99 latency <= L*", "unit": "requests/s",
                      "impl": "drk-serve", "data": "synthetic", "requests_per_run": nreq,
                      "saturation_frames_per_s": {m: v["frames_per_s"] for m, v in sat.items()},
                      "saturation_overlap": {m: v.get("overlap") for m, v in sat.items()},
                      "L_star_ms": L, "L_star_rule": "p99 of sequential rendering at half its saturation rate",
                      "max_rate": best, "runs": runs,
                      "config": {"scenes": [s.n for s in scenes], "resolutions": list(synth.SERVE_RESOLUTIONS),
                                 "weights": list(synth.SERVE_RES_WEIGHTS), "mem_budget": budget,
                                 "max_batch": args.serve_batch}}), flush=True)
    return 0


def main():
    args = parse()
    if args.serve_sweep:
        return serve_sweep(args)
    if args.serve:
        return run_serve(args)
    if args.order_study:
        return order_study(args)
    if args.train:
        return train_bench(args)
    if args.mesh:
        return mesh_bench(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_drk(args)


if __name__ == "__main__":
    sys.exit(main())
