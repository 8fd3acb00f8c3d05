#!/usr/bin/env python3
"""Benchmark: MERF baked-scene rendering on B300 (Mrays/s and 1080p frames/s vs the
feature-gather bandwidth roofline).

One step renders 8 cameras at 1920 x 1080 (16.6 M pixel rays) of the paper-scale synthetic
scene: 512^3 grid in 16^3 blocks, three 2048^2 planes, occupancy 128^3..16^3, step 1/256,
cameras on a ring of radius 1.5.  Inputs are resident in HBM before timing; the scene
(1442 MB on the device) and each step's output (199 MB) exceed the 126 MB L2, so no flush is
needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  `--impl reference` times the FP64 CPU oracle on host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s and 1080p frames/s vs gather-BW roofline; FP16 vs FP32 at PSNR>50 dB; p99 ms"
UNIT = "Mrays/s"
W_IMG, H_IMG, N_CAMS, STEP = 1920, 1080, 8, 1.0 / 256
WORKLOAD = ("paper-scale synthetic MERF scene (L=512 in 16^3 blocks, R=2048, uint8, occupancy "
            "128/64/32/16), 8 ring cameras (radius 1.5) at 1920x1080, lattice step 1/256, FP32 path")
# algorithmic gather bytes (no reuse): per evaluated sample 8 grid corners + 12 plane texels of
# the density byte (20 B) and one 4-byte index-grid entry; per sample with non-zero opacity the
# 7 appearance bytes of the same 20 texels (140 B); per ray the 12-byte RGB output.
B_DENSITY, B_INDEX, B_APPEAR, B_OUT = 20, 4, 140, 12


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one timed 8-camera render
# launch from an ncu capture of this workload; reported as roofline.traffic only while the
# render kernel's sources (device code, launch and scene layout) hash to the value they were
# measured with (otherwise null).
TRAFFIC_BYTES_PER_LAUNCH = (722.20 + 279.55) * 1e6
TRAFFIC_SOURCES = ("debug.cuh", "field.cuh", "geometry.h", "merf_api.cu", "render.cuh", "scene.h", "traverse.cuh",
                   "umma.cuh")
# Warp-level instructions (smsp__inst_executed.sum) of the same timed launch from an ncu capture
# (1 pass, full size), for the issue-rate roofline: the kernel is bound by instruction issue, and
# an SM's four schedulers issue at most one warp instruction per clock each.
INST_PER_LAUNCH = 34.947777282e9
SMS, SCHEDULERS_PER_SM = 148, 4
TRAFFIC_SOURCES_SHA256 = "3da0b7c1f60f5874bf95166a725e5e2043c3ac435f004b9c31a91cadb398c28d"


def _sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2302_12249_b300", "csrc")
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.path = index, None, None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 7:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        pw = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w": statistics.median(pw) if pw else None}


def _dist(backend: str = "nccl"):
    n = int(os.environ.get("WORLD_SIZE", "1"))
    if n > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
        return dist, int(os.environ["RANK"]), n, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


def _max_over_ranks(dist, value: float, device: str = "cuda") -> float:
    """The job's time is its slowest rank's: the maximum of `value` over the ranks."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_rate(rays_per_rank_step: int, world: int, steps: int, seconds: float) -> float:
    """Whole-job throughput in Mrays/s: every rank renders its own step (replicas, weak scaling),
    so the job processes world x rays per step in the slowest rank's time."""
    return rays_per_rank_step * world * steps / seconds / 1e6


def _oracle_leg(scene, cams):
    """The one part of the benchmark that runs the FP64 CPU oracle (host cores): the CPU
    baseline, the reference values the precision form is scored against, and the distinct data
    one 1080p frame reads (camera 0 of the workload, its own evaluated samples)."""
    import oracle
    osc = oracle.OracleScene(scene)
    cpu = _cpu_baseline(oracle, osc, cams)
    pcams, pix = _precision_pixels()
    lo = oracle.render(osc, pcams, W_IMG, H_IMG, STEP, pix=pix, t_term=2e-4 * 0.999)[:, 0:3]
    hi = oracle.render(osc, pcams, W_IMG, H_IMG, STEP, pix=pix, t_term=2e-4 * 1.001)[:, 0:3]
    t0 = time.perf_counter()
    fp = oracle.footprint(osc, cams[:1], W_IMG, H_IMG, STEP)
    fp["seconds"] = time.perf_counter() - t0
    return cpu, (pix, lo, hi), fp


def _cpu_baseline(oracle, osc, cams):
    """The FP64 oracle on the host cores: one full 1280x720 frame (camera 0 of the workload's
    ring at that resolution), and on one thread a ~3 s sample of random pixels of it."""
    from paper_2302_12249_b300 import synth
    threads = oracle.default_threads()
    W, H = 1280, 720
    cam = synth.config_cameras("paper", W=W, H=H)[:1]
    t0 = time.perf_counter()
    oracle.render(osc, cam, W, H, STEP, threads=threads)
    dt = time.perf_counter() - t0
    rng = np.random.default_rng(12345)
    rays1, t1 = 0, time.perf_counter()
    while time.perf_counter() - t1 < 3.0:
        n = 256
        pix = np.stack([np.zeros(n, int), rng.integers(0, W, n), rng.integers(0, H, n)], 1)
        oracle.render(osc, cam, W, H, STEP, pix=pix.astype(np.int32), threads=1)
        rays1 += n
    dt1 = time.perf_counter() - t1
    return {"value": W * H / dt / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"one full 1280x720 frame ({W * H} rays, {dt:.1f} s, FP64, {threads} threads)",
            "one_thread": {"value": rays1 / dt1 / 1e6, "unit": UNIT,
                           "sample": f"{rays1} random pixel rays of that frame ({dt1:.1f} s, FP64, 1 thread)"}}


def _frames_720p(gs, steps=10, warmup=3):
    """Frames/s at 1280x720 (the paper's other viewer resolution): the same 8 ring cameras and
    scene, FP32, CUDA-event time of `steps` launches after `warmup`."""
    import torch
    from paper_2302_12249_b300 import merf, synth
    W, H = 1280, 720
    cams = synth.config_cameras("paper", W=W, H=H)
    out = torch.empty((cams.shape[0], H, W, 3), dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        merf.render(gs, cams, W, H, STEP, out=out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        merf.render(gs, cams, W, H, STEP, out=out)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    return {"frames_per_s": cams.shape[0] / (ms / 1e3), "mrays_per_s": cams.shape[0] * W * H / (ms / 1e3) / 1e6,
            "ms_per_step": ms, "workload": f"{cams.shape[0]} ring cameras x {W}x{H}, FP32"}


PRECISION_CAMS, PRECISION_PIX = 64, 2000


def _precision_pixels():
    """The precision form's 64 ring cameras and the 2000 pixels its error is measured on."""
    from paper_2302_12249_b300 import synth
    cams = synth.ring_cameras(PRECISION_CAMS, W_IMG, H_IMG, radius=1.5, seed=synth.SEED_CAMERA + 1)
    rng = np.random.default_rng(99)
    pix = np.stack([rng.integers(0, PRECISION_CAMS, PRECISION_PIX), rng.integers(0, W_IMG, PRECISION_PIX),
                    rng.integers(0, H_IMG, PRECISION_PIX)], 1).astype(np.int32)
    return cams, pix


def _precision_form(gs, ref=None, steps=3):
    """Precision form: the same scene rendered from 64 ring cameras at 1920x1080 in FP32, FP16 and
    BF16 (uint8 features, appearance arithmetic and deferred MLP in 16 bits on tensor cores,
    density/transmittance/compositing in FP32).  Time per step and, on sampled pixels, the
    error against the FP64 oracle (max |dRGB| per channel and PSNR) when the oracle leg supplied
    its reference values `ref` = (pixels, lower, upper threshold renders)."""
    import torch
    from paper_2302_12249_b300 import merf
    cams, pix = _precision_pixels()
    n_cams, n_pix = cams.shape[0], pix.shape[0]
    out = torch.empty((n_cams, H_IMG, W_IMG, 3), dtype=torch.float32, device="cuda")
    lin = torch.from_numpy((pix[:, 0].astype(np.int64) * H_IMG + pix[:, 2]) * W_IMG + pix[:, 1]).cuda()
    res = {}
    for name, prec in (("fp32", merf.PREC_FP32), ("fp16", merf.PREC_FP16), ("bf16", merf.PREC_BF16)):
        merf.render(gs, cams, W_IMG, H_IMG, STEP, out=out, precision=prec)
        torch.cuda.synchronize()
        ck = Clocks(torch.cuda.current_device())
        ck.start()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            merf.render(gs, cams, W_IMG, H_IMG, STEP, out=out, precision=prec)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        res[name] = {"ms_per_step": ms, "mrays_per_s": n_cams * W_IMG * H_IMG / (ms / 1e3) / 1e6,
                     "clocks": ck.stop()}
        if ref is not None:
            _, lo, hi = ref
            rgb = out.reshape(-1, 3)[lin].double().cpu().numpy()
            e_lo, e_hi = np.abs(rgb - lo).max(axis=1), np.abs(rgb - hi).max(axis=1)
            closest = np.where((e_lo <= e_hi)[:, None], lo, hi)
            mse = float(np.mean((rgb - closest) ** 2))
            res[name]["max_abs_err"] = float(np.abs(rgb - closest).max())
            res[name]["psnr_db"] = (10 * math.log10(1.0 / mse)) if mse > 0 else None
    res["workload"] = f"{n_cams} ring cameras x 1920x1080, {steps} timed steps each; error on {n_pix} sampled pixels"
    res["fp16_speedup_vs_fp32"] = res["fp32"]["ms_per_step"] / res["fp16"]["ms_per_step"]
    return res


def _differentiation(steps: int = 5):
    """Differentiation form: dense float scene (128^3 grid, 512^2 planes), 4 cameras at 512x512,
    L2 loss against a seeded target; forward, then the hand-written adjoint through autograd."""
    import torch
    from paper_2302_12249_b300 import merf, synth
    sc = synth.make_scene("dense128")
    gs = merf.Scene(sc)
    cams = synth.config_cameras("dense128")
    grid = torch.from_numpy(sc.grid_f32).cuda().requires_grad_(True)
    planes = torch.from_numpy(sc.planes_f32).cuda().requires_grad_(True)
    mlp = torch.from_numpy(sc.mlp).cuda().requires_grad_(True)
    target = torch.rand((4, 512, 512, 3), generator=torch.Generator().manual_seed(5)).cuda()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd = bwd = 0.0
    for it in range(steps + 2):
        grid.grad = planes.grad = mlp.grad = None
        ev[0].record()
        out = merf.render_differentiable(gs, grid, planes, mlp, cams, 512, 512, sc.cfg.step)
        loss = 0.5 * ((out - target) ** 2).sum()
        ev[1].record()
        loss.backward()
        ev[2].record()
        torch.cuda.synchronize()
        if it >= 2:
            fwd += ev[0].elapsed_time(ev[1])
            bwd += ev[1].elapsed_time(ev[2])
    rays = 4 * 512 * 512
    gs.close()
    return {"workload": "dense float 128^3 grid + 3 x 512^2 planes, 4 cameras x 512x512, L2 loss",
            "forward_ms": fwd / steps, "backward_ms": bwd / steps,
            "backward_mrays_per_s": rays / (bwd / steps / 1e3) / 1e6}


def _grid_only_variant(merf_ref, names=("snerg512", "snerg1024", "snerg2048"), steps=5, warmup=3):
    """The SNeRG++-style baseline the paper compares MERF with (Sec. 6): the same contents baked
    as a grid-only scene (no planes) at L = 512, 1024 and 2048 (the paper's SNeRG++ default),
    rendered by the same kernel from the same 8 cameras at 1920x1080 in FP32.  L = 2048 bakes
    about 28 GB of stored blocks: they are generated on the GPU and uploaded from device memory
    (merf_scene_upload_device).  Per configuration: device memory (the library's layout: texel
    pairs, about twice the baked arrays) and the baked arrays' size, time, Mrays/s and the
    algorithmic gather bytes (per evaluated sample 8 density bytes + the 4-byte index entry, per
    sample with non-zero opacity 56 appearance bytes, per ray 12 output bytes)."""
    import torch
    from paper_2302_12249_b300 import merf, synth
    cams = synth.config_cameras("paper")
    n = cams.shape[0]
    res = {"merf": merf_ref}
    for name in names:
        t_build = time.perf_counter()
        sc = synth.make_scene(name, device="cuda" if synth.CONFIGS[name].L >= 2048 else "cpu")
        baked = sc.baked_bytes()
        gs = merf.Scene(sc)
        if torch.is_tensor(sc.atlas):
            sc.atlas = None                  # the library holds its own padded copy
            torch.cuda.empty_cache()
        t_build = time.perf_counter() - t_build
        out = torch.empty((n, H_IMG, W_IMG, 3), dtype=torch.float32, device="cuda")
        cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
        aux = torch.empty((n, H_IMG, W_IMG, merf.AUX_SIZE), dtype=torch.float32, device="cuda")
        merf.render(gs, cams, W_IMG, H_IMG, STEP, out=out, aux=aux, counters=cnt)
        torch.cuda.synchronize()
        del aux
        c = [int(v) for v in cnt.cpu().tolist()]
        for _ in range(warmup):
            merf.render(gs, cams, W_IMG, H_IMG, STEP, out=out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            merf.render(gs, cams, W_IMG, H_IMG, STEP, out=out)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        alg = c[merf.CNT_EVAL] * (8 + B_INDEX) + c[merf.CNT_APPEAR] * 56 + c[merf.CNT_RAYS] * B_OUT
        res[name] = {"L": sc.cfg.L, "device_mb": round(gs.device_bytes / 1e6, 1), "baked_mb": round(baked / 1e6, 1),
                     "ms_per_step": ms, "build_s": round(t_build, 1),
                     "mrays_per_s": n * W_IMG * H_IMG / (ms / 1e3) / 1e6,
                     "evaluated_per_ray": c[merf.CNT_EVAL] / c[merf.CNT_RAYS],
                     "gather_bytes_per_sample": 8 + B_INDEX + 56,
                     "algorithmic_gb_per_s": alg / (ms / 1e3) / 1e9}
        gs.close()
        del sc, out
    res["workload"] = ("same contents as grid-only scenes (3D grid alone, 16^3 blocks, no planes), the 8 ring "
                       "cameras at 1920x1080, FP32; `merf` is this run's main line")
    return res


def _sparse_scene(steps=5, warmup=3):
    """The paper-scale configuration at the sparsity and size of the paper's scenes: the same 256
    blobs with radii U(0.01, 0.08), about 9 % of 16^3 blocks stored (the configured scene stores
    48 %), and its grid-only (SNeRG++-style) counterpart at L = 2048, the same 8 cameras at
    1920x1080 in FP32: device memory and baked size, time, Mrays/s and evaluated samples per ray."""
    import torch
    from paper_2302_12249_b300 import merf, synth
    cams = synth.config_cameras("paper")
    n = cams.shape[0]
    res = {}
    for name in ("paper_sparse", "snerg2048_sparse"):
        cfg = synth.CONFIGS[name]
        sc = synth.make_scene(name, device="cuda" if cfg.grid_only else "cpu")
        baked = sc.baked_bytes()
        gs = merf.Scene(sc)
        if torch.is_tensor(sc.atlas):
            sc.atlas = None
            torch.cuda.empty_cache()
        out = torch.empty((n, H_IMG, W_IMG, 3), dtype=torch.float32, device="cuda")
        cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
        merf.render(gs, cams, W_IMG, H_IMG, STEP, out=out, counters=cnt)
        for _ in range(warmup):
            merf.render(gs, cams, W_IMG, H_IMG, STEP, out=out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            merf.render(gs, cams, W_IMG, H_IMG, STEP, out=out)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        c = [int(v) for v in cnt.cpu().tolist()]
        res[name] = {"L": cfg.L, "R": cfg.R, "block_fraction": round(sc.stats["block_fraction"], 4),
                     "device_mb": round(gs.device_bytes / 1e6, 1), "baked_mb": round(baked / 1e6, 1),
                     "ms_per_step": ms, "mrays_per_s": n * W_IMG * H_IMG / (ms / 1e3) / 1e6,
                     "evaluated_per_ray": c[merf.CNT_EVAL] / c[merf.CNT_RAYS]}
        gs.close()
        del sc, out
    res["memory_ratio_grid_only_to_merf"] = res["snerg2048_sparse"]["device_mb"] / res["paper_sparse"]["device_mb"]
    res["baked_ratio_grid_only_to_merf"] = res["snerg2048_sparse"]["baked_mb"] / res["paper_sparse"]["baked_mb"]
    res["workload"] = ("paper-scale scene with blob radii U(0.01, 0.08) (256 blobs, half in the unit cube), MERF "
                       "L=512 + three 2048^2 planes and grid-only L=2048, the 8 ring cameras at 1920x1080, FP32")
    return res


def _spherical_ablation(gs, merf_ref, steps=5, warmup=3):
    """The ablation of Sec. 3.2 / Table 2 (c): the same scene and cameras rendered with mip-NeRF
    360's spherical contraction, which bends rays so nothing can be skipped -- every sample of a
    dense march is visited and its own finest occupancy cell tested (FP32).  Reports the time,
    the visited and evaluated samples per ray and the slowdown against contract_pi."""
    import torch
    from paper_2302_12249_b300 import merf, synth
    cams = synth.config_cameras("paper")
    n = cams.shape[0]
    out = torch.empty((n, H_IMG, W_IMG, 3), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    aux = torch.empty((n, H_IMG, W_IMG, merf.AUX_SIZE), dtype=torch.float32, device="cuda")
    merf.render(gs, cams, W_IMG, H_IMG, STEP, out=out, aux=aux, counters=cnt, contraction=merf.CONTRACT_SPHERICAL)
    torch.cuda.synchronize()
    del aux
    c = [int(v) for v in cnt.cpu().tolist()]
    for _ in range(warmup):
        merf.render(gs, cams, W_IMG, H_IMG, STEP, out=out, contraction=merf.CONTRACT_SPHERICAL)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        merf.render(gs, cams, W_IMG, H_IMG, STEP, out=out, contraction=merf.CONTRACT_SPHERICAL)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    return {"ms_per_step": ms, "mrays_per_s": n * W_IMG * H_IMG / (ms / 1e3) / 1e6,
            "visited_per_ray": c[merf.CNT_LATTICE] / c[merf.CNT_RAYS],
            "evaluated_per_ray": c[merf.CNT_EVAL] / c[merf.CNT_RAYS],
            "contract_pi": {"ms_per_step": merf_ref["ms_per_step"], "mrays_per_s": merf_ref["mrays_per_s"],
                            "lattice_per_ray": merf_ref["lattice_per_ray"],
                            "evaluated_per_ray": merf_ref["evaluated_per_ray"]},
            "slowdown": ms / merf_ref["ms_per_step"],
            "workload": "paper-scale scene, the 8 ring cameras at 1920x1080, FP32, spherical contraction "
                        "marched densely (samples uniform in s, t(s) = s then 1/(2 - s))"}


SERVE_RES = [(256, 256), (640, 360), (1280, 720), (1920, 1080)]


def _serving_stream(srv, n_scenes: int, n_requests: int, rate, seed_arrivals: int, bufs) -> dict:
    """One request stream through a running server.  rate: Poisson arrivals per second, or None for
    saturation (every request offered at once; in flight as many as the host buffers allow).
    Returns latency percentiles overall and per resolution, and where the latency went
    (merf_request_timing: admission, queue, render, copy-back), for all requests and for the
    slowest 1 %."""
    import queue
    import threading
    from paper_2302_12249_b300 import synth
    rng = np.random.default_rng(seed_arrivals)
    gaps = rng.exponential(1.0 / rate, size=n_requests) if rate else np.zeros(n_requests)
    which = rng.integers(0, n_scenes, size=n_requests)
    res = rng.integers(0, len(SERVE_RES), size=n_requests)
    radius = rng.uniform(1.2, 3.0, size=n_requests)
    az = rng.uniform(0, 2 * math.pi, size=n_requests)
    el = np.radians(rng.uniform(-30, 30, size=n_requests))
    submitted = queue.Queue()
    phases = ("admit_s", "queue_s", "render_s", "copy_s")
    lat = np.zeros(n_requests)
    part = np.zeros((n_requests, len(phases)))
    lags = np.zeros(n_requests)
    blocked = [0]

    def collector():
        for k in range(n_requests):
            rid, r, b = submitted.get()
            t = srv.wait_timed(rid, timeout=600.0)
            lat[k] = t["total_s"]
            part[k] = [t[p] for p in phases]
            bufs[r].put(b)

    th = threading.Thread(target=collector)
    th.start()
    t0 = time.perf_counter()
    t_next = t0
    for k in range(n_requests):
        t_next += gaps[k]
        dt = t_next - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        lags[k] = time.perf_counter() - t_next
        r = int(res[k])
        W, H = SERVE_RES[r]
        if bufs[r].empty():
            blocked[0] += 1
        b = bufs[r].get()
        eye = radius[k] * np.array([math.cos(el[k]) * math.cos(az[k]), math.cos(el[k]) * math.sin(az[k]), math.sin(el[k])])
        cam = synth.camera_record(synth.look_at(eye), W, H)
        submitted.put((srv.submit(int(which[k]), cam, W, H, b), r, b))
    th.join()
    t_end = time.perf_counter()
    rays = sum(SERVE_RES[int(r)][0] * SERVE_RES[int(r)][1] for r in res)
    ms = lambda v: float(v * 1e3)
    per_res = {}
    for r, (W, H) in enumerate(SERVE_RES):
        sel = res == r
        if sel.any():
            per_res[f"{W}x{H}"] = {"count": int(sel.sum()), "p50_ms": ms(np.percentile(lat[sel], 50)),
                                   "p99_ms": ms(np.percentile(lat[sel], 99)),
                                   "mean_render_ms": ms(part[sel, 2].mean())}
    tail = lat >= np.percentile(lat, 99)
    out = {"requests": n_requests, "arrival_rate_per_s": rate if rate else "saturation",
           "p50_ms": ms(np.percentile(lat, 50)), "p99_ms": ms(np.percentile(lat, 99)),
           "mean_ms": ms(lat.mean()), "max_ms": ms(lat.max()),
           "aggregate_mrays_per_s": rays / (t_end - t0) / 1e6,
           "offered_mrays_per_s": (rays / gaps.sum() / 1e6) if rate else None,
           "wall_s": t_end - t0, "per_resolution": per_res,
           "phases_mean_ms": {p[:-2]: ms(part[:, i].mean()) for i, p in enumerate(phases)},
           "phases_p99_ms": {p[:-2]: ms(np.percentile(part[:, i], 99)) for i, p in enumerate(phases)},
           "slowest_1pct_phases_mean_ms": {p[:-2]: ms(part[tail, i].mean()) for i, p in enumerate(phases)},
           "slowest_1pct_resolutions": {f"{W}x{H}": int((res[tail] == r).sum()) for r, (W, H) in enumerate(SERVE_RES)},
           "submit_lag_p99_ms": ms(np.percentile(lags, 99)), "host_buffer_waits": blocked[0]}
    return out


def _serving(gs_first, n_requests: int, rate: float = 200.0, seed_arrivals: int = 4000, max_tiles: int = 16384,
             max_tiles_backlog: int = 65536, sweep=((300.0, 4000), (400.0, 4000), (None, 2000))):
    """Serving form: four resident paper-scale scenes, Poisson arrivals, random scene and orbit
    camera, resolution uniform over SERVE_RES, FP16 continuous batching.  Latency is measured by the
    library from submission to the image being in host memory.  The configured stream (200
    requests/s) first, then a sweep of higher rates and saturation on the same server."""
    import queue
    import torch
    from paper_2302_12249_b300 import merf, synth
    scenes = [gs_first] + [merf.Scene(synth.make_scene("paper", seed=synth.SEED_SCENE + k)) for k in (1, 2, 3)]
    free_b, total_b = torch.cuda.mem_get_info()
    pool = int(min(4 << 30, free_b // 4))
    srv = merf.Server(scenes, pool_bytes=pool, step=STEP, max_tiles_per_iter=max_tiles, precision=merf.PREC_FP16,
                      max_tiles_backlog=max_tiles_backlog)
    bufs = {r: queue.Queue() for r in range(len(SERVE_RES))}
    for r, (W, H) in enumerate(SERVE_RES):
        for _ in range(48):
            bufs[r].put(torch.empty((H, W, 3), dtype=torch.float32, pin_memory=True))
    # warm-up: one request per resolution
    for r, (W, H) in enumerate(SERVE_RES):
        b = bufs[r].get()
        cam = synth.camera_record(synth.look_at([2.0, 0.0, 0.3]), W, H)
        srv.wait(srv.submit(0, cam, W, H, b))
        bufs[r].put(b)
    it0 = srv.stats()["iterations"]
    main = _serving_stream(srv, len(scenes), n_requests, rate, seed_arrivals, bufs)
    st = srv.stats()
    runs = []
    for k, (r, n) in enumerate(sweep):
        runs.append(_serving_stream(srv, len(scenes), n, r, seed_arrivals + 1 + k, bufs))
    srv.close()
    for sc in scenes[1:]:
        sc.close()
    main.update({"precision": "fp16", "max_tiles_per_iter": max_tiles, "max_tiles_backlog": max_tiles_backlog,
                 "iterations": st["iterations"] - it0,
                 "peak_admitted": st["peak_admitted"], "pool_mb": st["pool_bytes"] / 1e6,
                 "peak_pool_mb": st["peak_pool_bytes"] / 1e6,
                 "sweep": runs,
                 "workload": "4 resident paper-scale scenes (seeds 1000-1003), Poisson arrivals, random scene and "
                             "orbit (radius U(1.2,3), elevation U(-30,30) deg), resolution uniform over "
                             "256x256/640x360/1280x720/1920x1080; latency = submit to image in host memory, split "
                             "into admission (pool memory), queue (to the first launch of its tiles), render (to "
                             "the end of its last iteration) and copy-back; sweep: 300 and 400 requests/s and "
                             "saturation (every request offered at once, at most 48 in flight per resolution)"})
    return main


def run_reference(args):
    dist, rank, world, _ = _dist()
    if rank != 0:
        return 0
    from paper_2302_12249_b300 import synth
    import oracle
    scene = synth.make_scene("paper")
    cams = synth.config_cameras("paper")
    osc = oracle.OracleScene(scene)
    threads = oracle.default_threads()
    rng = np.random.default_rng(777)
    per_step = 4096
    samples = [np.stack([rng.integers(0, N_CAMS, per_step), rng.integers(0, W_IMG, per_step),
                         rng.integers(0, H_IMG, per_step)], 1).astype(np.int32)
               for _ in range(args.warmup + args.steps)]
    for s in range(args.warmup):
        oracle.render(osc, cams, W_IMG, H_IMG, STEP, pix=samples[s], threads=threads)
    t0 = time.perf_counter()
    for s in range(args.steps):
        oracle.render(osc, cams, W_IMG, H_IMG, STEP, pix=samples[args.warmup + s], threads=threads)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD.replace("FP32 path", "FP64 oracle") +
                                   "; each step renders 4096 random pixel rays of it",
                       "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} random pixel rays per step, FP64 oracle, {threads} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    dist, rank, world, local = _dist()
    torch.cuda.set_device(local)
    from paper_2302_12249_b300 import merf, synth
    scene = synth.make_scene("paper")
    cams = synth.config_cameras("paper")
    gs = merf.Scene(scene)
    cams = cams[:args.cams]
    n_cams = cams.shape[0]
    rays_per_step = n_cams * W_IMG * H_IMG
    prec = {"fp32": merf.PREC_FP32, "fp16": merf.PREC_FP16, "bf16": merf.PREC_BF16}[args.precision]
    out = torch.empty((n_cams, H_IMG, W_IMG, 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # untimed pass with counters: units of work per launch for the algorithmic byte count
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    aux = torch.empty((n_cams, H_IMG, W_IMG, merf.AUX_SIZE), dtype=torch.float32, device="cuda")
    merf.render(gs, cams, W_IMG, H_IMG, STEP, out=out, aux=aux, counters=cnt, precision=prec)
    torch.cuda.synchronize()
    c = [int(v) for v in cnt.cpu().tolist()]
    del aux
    alg_bytes = (c[merf.CNT_EVAL] * (B_DENSITY + B_INDEX) + c[merf.CNT_APPEAR] * B_APPEAR +
                 c[merf.CNT_RAYS] * B_OUT)

    for _ in range(args.warmup):
        merf.render(gs, cams, W_IMG, H_IMG, STEP, out=out, precision=prec)
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(args.steps):
        ev[s][0].record(stream)
        merf.render(gs, cams, W_IMG, H_IMG, STEP, out=out, precision=prec)
        ev[s][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    kern_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = _max_over_ranks(dist, total_ms)
    ms_per_step = total_ms / args.steps
    value = _job_rate(rays_per_step, world, args.steps, total_ms / 1e3)
    mean_kern_ms = sum(kern_ms) / len(kern_ms)
    peak, peak_src = _peaks()
    achieved = alg_bytes / (mean_kern_ms / 1e3) / 1e9

    # end to end through the host-output entry point: camera records in, RGB frames out
    e2e = None
    if not args.no_e2e:
        staging = torch.empty_like(out)
        host = torch.empty(out.shape, dtype=torch.float32, pin_memory=True)
        merf.render_host(gs, cams, W_IMG, H_IMG, STEP, staging, host, precision=prec)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            merf.render_host(gs, cams, W_IMG, H_IMG, STEP, staging, host, precision=prec)
        e2e_s = time.perf_counter() - t0
        e2e_s = _max_over_ranks(dist, e2e_s)
        e2e = {"value": _job_rate(rays_per_step, world, args.steps, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": n_cams * 64, "d2h_bytes_per_step": int(out.numel() * 4)}

    p720 = None
    if rank == 0 and world == 1 and not args.no_precision:
        p720 = _frames_720p(gs)
    cpu = prec_ref = footprint = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, prec_ref, footprint = _oracle_leg(scene, synth.config_cameras("paper"))
    precision = None
    if rank == 0 and world == 1 and not args.no_precision:
        precision = _precision_form(gs, prec_ref)
    differentiation = None
    if rank == 0 and world == 1 and not args.no_diff:
        differentiation = _differentiation()
    serving = None
    if rank == 0 and world == 1 and args.serve_requests > 0:
        serving = _serving(gs, args.serve_requests)
    variants = ablation = sparse = None
    if rank == 0 and world == 1 and not args.no_variants:
        merf_ref = {"L": 512, "R": 2048, "device_mb": round(gs.device_bytes / 1e6, 1),
                    "baked_mb": round(scene.baked_bytes() / 1e6, 1), "ms_per_step": ms_per_step,
                    "mrays_per_s": value, "evaluated_per_ray": c[merf.CNT_EVAL] / c[merf.CNT_RAYS],
                    "gather_bytes_per_sample": B_DENSITY + B_INDEX + B_APPEAR,
                    "algorithmic_gb_per_s": achieved}
        ablation = _spherical_ablation(gs, dict(merf_ref, lattice_per_ray=c[merf.CNT_LATTICE] / c[merf.CNT_RAYS]))
        variants = _grid_only_variant(merf_ref)
        sparse = _sparse_scene()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"fp32": "f32", "fp16": "f16", "bf16": "bf16"}[args.precision],
                "data": "synthetic",
                "config": {"workload": WORKLOAD.replace("FP32 path", f"{args.precision.upper()} path"),
                           "rays_per_step_per_gpu": rays_per_step,
                           "scene_device_mb": round(gs.device_bytes / 1e6, 1),
                           "scene_baked_mb": round(scene.baked_bytes() / 1e6, 1),
                           "block_fraction": round(scene.stats["block_fraction"], 4),
                           "l2": "inputs larger than L2 (scene and per-step output each exceed 126 MB); no flush",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "frames_per_s_1080p": value * 1e6 / (W_IMG * H_IMG),
                "step_ms": {"mean": mean_kern_ms, "median": statistics.median(kern_ms), "min": min(kern_ms),
                            "max": max(kern_ms), "frames": n_cams * args.steps},
                "work": {"lattice_per_ray": c[merf.CNT_LATTICE] / c[merf.CNT_RAYS],
                         "evaluated_per_ray": c[merf.CNT_EVAL] / c[merf.CNT_RAYS],
                         "appearance_per_ray": c[merf.CNT_APPEAR] / c[merf.CNT_RAYS],
                         "algorithmic_bytes_per_ray": alg_bytes / c[merf.CNT_RAYS]},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak,
                             "traffic": (TRAFFIC_BYTES_PER_LAUNCH
                                         if _sources_sha256() == TRAFFIC_SOURCES_SHA256 and n_cams == N_CAMS
                                         and args.precision == "fp32" else None),
                             "kernel": f"render_kernel<0,{prec},1,0> ({args.precision.upper()})",
                             "kernel_ms": mean_kern_ms,
                             "peak_source": peak_src,
                             "note": "algorithmic gather bytes (no reuse) over the measured HBM copy peak, as "
                                     "the metric defines its roofline; L1/L2 serve all but 0.3 % of the "
                                     "gather, and the binding limit is instruction issue (roofline_issue)"},
                "gpu_launches": args.steps,
                "e2e": e2e, "clocks": ck}
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if (line["roofline"]["traffic"] is not None and ck and ck.get("sm_mhz")):
            issue = INST_PER_LAUNCH / (mean_kern_ms / 1e3) / 1e9
            peak_issue = SMS * SCHEDULERS_PER_SM * ck["sm_mhz"] / 1e3
            line["roofline_issue"] = {"bound": "issue", "achieved": issue, "peak": peak_issue, "unit": "Ginst/s",
                                      "frac": issue / peak_issue, "inst_per_launch": INST_PER_LAUNCH,
                                      "peak_from": f"{SMS} SMs x {SCHEDULERS_PER_SM} schedulers x 1 warp "
                                                   f"instruction per clock at the sampled {ck['sm_mhz']:.0f} MHz"}
        if footprint is not None:
            line["footprint_1080p_frame"] = dict(
                footprint, algorithmic_bytes=alg_bytes / n_cams,
                dram_bytes=(TRAFFIC_BYTES_PER_LAUNCH / N_CAMS if line["roofline"]["traffic"] else None),
                frame="camera 0 of the workload, its evaluated samples, counted by the FP64 oracle")
        if p720 is not None:
            line["frames_720p"] = p720
        if precision is not None:
            line["precision_form"] = precision
        if differentiation is not None:
            line["differentiation"] = differentiation
        if serving is not None:
            line["serving"] = serving
        if variants is not None:
            line["grid_only_variant"] = variants
        if ablation is not None:
            line["spherical_ablation"] = ablation
        if sparse is not None:
            line["paper_sparsity_scene"] = sparse
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cams", type=int, default=N_CAMS, help="cameras per step (profiling cases)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-output measurement (profiling)")
    ap.add_argument("--no-precision", action="store_true", help="skip the FP16/BF16 comparison (profiling)")
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiation form (profiling)")
    ap.add_argument("--serve-requests", type=int, default=10000, help="requests of the serving run (0 = skip)")
    ap.add_argument("--no-variants", action="store_true", help="skip the grid-only comparison (profiling)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16"],
                    help="arithmetic of the main line (default FP32; the precision form is also reported)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
