#!/usr/bin/env python
"""Throughput of disk-blended light field rendering of stereo eye views.

Workload (default): the rig-scale light field - 24 textured spheres in a
backdrop, 1,024 source views of 1024x1024 (120 degrees) spread over a capture
sphere of radius 0.35 m, 64x64 per-view meshes, FP32 RGBA textures resident
in HBM - rendered as a stereo pair of 1440x1600 eye views (IPD 64 mm) per
step, cycling through seeded random head poses.  A step is one lf_render call
for both eyes.  L2 is flushed (a 256 MiB write) between steps, outside the
timed events.

Prints one JSON line.  `--impl reference` times the CPU oracle instead (the
reference arm: the plain FP64 restatement of the method on the host cores),
on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "output Mpix/s (stereo eye views) vs plain FP32 form; % texel-fetch HBM roofline"
UNIT = "Mpix/s"
HBM_FALLBACK_GBS = 6800.0


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    # the default workload is the rig-scale stereo frame; "batch" is the 128-eye batched form
    p.add_argument("--steps", type=int, default=None,
                   help="timed steps [rig: 2000, batch: 60, others: 400], about a second of timed device "
                        "work so the clock sampler sees the load")
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["rig", "rig256", "tiny", "batch", "learned", "refine", "train",
                                          "prefilter", "twolevel"],
                   default="rig")
    p.add_argument("--samples", type=int, default=32, help="prefilter: Monte Carlo samples per pixel (Eq. 5)")
    p.add_argument("--supersample", type=int, default=1, help="prefilter: scale of the Lbar renders")
    p.add_argument("--refine-kernel", choices=["fused", "layers"], default="fused")
    p.add_argument("--poses", type=int, default=8, help="distinct head poses cycled through")
    p.add_argument("--tex", choices=["f32", "u8", "bf16", "fp8"], default="f32")
    p.add_argument("--mesh", choices=["f32", "f16"], default="f32")
    p.add_argument("--disk", choices=["round", "oval"], default="round",
                   help="round disks on the capture sphere, or asymmetric ovals sized by the Delaunay 1-ring")
    p.add_argument("--quality-pixels", type=int, default=3000,
                   help="random pixels per eye compared with the FP64 oracle (0 to skip)")
    p.add_argument("--tile", default="16x16")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="bound on the CPU baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip the batched, reduced-precision and learned forms")
    p.add_argument("--pages", type=int, default=256, help="twolevel: device pages of the fine level")
    p.add_argument("--budget", type=int, default=32, help="twolevel: page uploads per frame")
    p.add_argument("--save-refiner", default=None, help="learned: write the trained weights and their quality here")
    # learned refinement workload
    p.add_argument("--pairs", type=int, default=4096, help="learned: 256x256 training crops")
    p.add_argument("--train-steps", type=int, default=1500, help="learned: Adam steps (batch 16)")
    p.add_argument("--eval-eyes", type=int, default=128, help="learned: held-out 1440x1600 eyes")
    p.add_argument("--dense-views", type=int, default=4096)
    p.add_argument("--dense-grid", type=int, default=256)
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world: int):
    """One process per GPU under torchrun (NCCL), or gloo ranks on the CPU."""
    if world > 1:
        import torch
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")


def finish_dist(world: int):
    if world > 1:
        import torch.distributed as dist

        if dist.is_initialized():
            dist.destroy_process_group()


def max_over_ranks(ms: float) -> float:
    """The slowest rank's duration (the job's time); the value itself at N = 1.
    Ranks render independent head poses (replicas): no data crosses ranks."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier_all():
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def whole_job_rate(units_per_rank: float, max_ms: float, world: int) -> float:
    """Units all ranks processed per second (millions), over the slowest rank's time."""
    return world * units_per_rank / (max_ms / 1000.0) / 1e6


def make_workload(name: str, n_heads: int, rank: int):
    import scene

    if name == "tiny":
        lf = scene.tiny_light_field(1)
        rng = scene.SplitMix64(1000 + rank)
        import math as m
        lf.eyes = []
        for _ in range(n_heads):
            lf.eyes += scene.head_pose_eyes(rng, 256, 256, 90.0, yaw_range=(-m.radians(10), m.radians(10)),
                                            pitch_deg=10.0)
        desc = ("tiny cap: 8 spheres, 16 views 128x128 (90 deg) on a 40 deg cap, 32x32 meshes, "
                "stereo 2x256x256 eyes")
    else:
        src = 1024 if name == "rig" else 256
        lf = scene.rig_light_field(1, width=src, n_heads=0)
        rng = scene.SplitMix64(29 + 7919 + 104729 * rank)
        for _ in range(n_heads):
            lf.eyes += scene.head_pose_eyes(rng, 1440, 1600, 100.0)
        desc = ("rig scale: 24 spheres, 1024 Fibonacci views %dx%d (120 deg) on a 0.35 m sphere, "
                "64x64 meshes, stereo 2x1440x1600 eyes (100 deg, IPD 64 mm)" % (src, src))
    heads = [lf.eyes[2 * k:2 * k + 2] for k in range(n_heads)]
    return lf, heads, desc


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


RASTER_SOURCES = ("lf_raster.cu", "lf_internal.h")
REFINE_SOURCES = ("lf_refine_tc.cu", "lf_internal.h")
REFINE_PROFILE = "refine_fused_stereo_2x1440x1600"


def kernel_source_hash(files=RASTER_SOURCES) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1810_08860_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


E2E_WHAT = ("%s: host poses in, %s delivered to pinned host memory by the context's copy stream while "
            "the next frame renders; wall clock over the run, with the 256 MiB L2 flush before each frame "
            "inside it; frame_latency_ms: one frame at a time, call to delivery")


def host_memory_available() -> int:
    """Bytes of host memory this process may still use: the smaller of the
    kernel's MemAvailable and the cgroup's remaining limit (0 if unknown)."""
    avail = 0
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        return 0
    try:
        with open("/sys/fs/cgroup/memory.max") as fh:
            lim = fh.read().strip()
        if lim != "max":
            with open("/sys/fs/cgroup/memory.current") as fh:
                avail = min(avail, int(lim) - int(fh.read().strip()))
    except (OSError, ValueError):
        pass
    return max(avail, 0)


def host_e2e(r, heads, shapes, flush, stream, steps, px_per_step, world, form="plain", in_flight=None):
    """Whole-job throughput of lf_render_host over `steps` pipelined frames
    (wall clock, max over ranks) and the mean single-frame latency.  At most
    `in_flight` frames are undelivered at a time, each with its own pinned
    host images (default: as many as the library pipelines)."""
    import torch
    import paper_1810_08860_gb300 as lfm

    n_sets = in_flight or lfm.HOST_FRAMES_IN_FLIGHT
    sets = [[torch.empty(sh, dtype=torch.float32, pin_memory=True) for sh in shapes] for _ in range(n_sets)]
    for k in range(lfm.HOST_FRAMES_IN_FLIGHT):  # allocate every device slot of the library before timing
        r.render_host(heads[k % len(heads)], out=sets[k % n_sets], form=form, stream=stream)
        r.host_wait()
    torch.cuda.synchronize()
    barrier_all()
    t0 = time.perf_counter()
    issued = []
    for k in range(steps):
        if k >= n_sets:
            r.host_wait(issued[k - n_sets])  # its host images are about to be reused
        flush.zero_()
        f, _ = r.render_host(heads[k % len(heads)], out=sets[k % len(sets)], form=form, stream=stream)
        issued.append(f)
    if r.host_wait() != 0:
        raise RuntimeError("a frame delivered to host memory reported device errors")
    total_ms = max_over_ranks(1000.0 * (time.perf_counter() - t0))
    lat = []
    for k in range(min(steps, 50)):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        f, _ = r.render_host(heads[k % len(heads)], out=sets[0], form=form, stream=stream)
        r.host_wait(f)
        lat.append(1000.0 * (time.perf_counter() - t1))
    return whole_job_rate(px_per_step * steps, total_ms, world), statistics.mean(lat)


def ncu_value(profile: str, key: str, files=RASTER_SOURCES):
    """A figure from the committed ncu summary profiles/<profile>.txt, if it was
    taken on the current source of the kernel (`files`); else None."""
    path = os.path.join(ROOT, "profiles", profile + ".txt")
    try:
        vals = {}
        with open(path) as fh:
            for line in fh:
                if ":" in line:
                    k, v = line.split(":", 1)
                    vals[k.strip()] = v.strip()
        if vals.get("kernel_source_sha") != kernel_source_hash(files):
            return None
        return float(vals[key])
    except Exception:
        return None


def ncu_traffic(profile: str, files=RASTER_SOURCES):
    """DRAM bytes per launch from the committed ncu summary (see ncu_value)."""
    return ncu_value(profile, "dram_bytes_per_launch", files)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for n, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(lf, eye, seconds: float):
    """The oracle, as it stands, on the host cores: Mpix/s over a bounded
    sample of random pixels of one eye of the workload."""
    import numpy as np

    import oracle

    cores = os.cpu_count() or 1
    rng = np.random.default_rng(7)
    n = 2000
    total_pix, total_t = 0, 0.0
    while True:
        pix = np.stack([rng.integers(0, eye.width, n), rng.integers(0, eye.height, n)], axis=1)
        t0 = time.perf_counter()
        oracle.render(lf, eye, pixels=pix, threads=cores)
        dt = time.perf_counter() - t0
        total_pix += n
        total_t += dt
        if total_t >= seconds or total_pix >= 4_000_000:
            break
        n = int(min(max(n * 2, 2000), 400_000))
    # the same oracle on one thread, over a smaller bounded sample
    n1, t1 = 2000, 0.0
    pix = np.stack([rng.integers(0, eye.width, n1), rng.integers(0, eye.height, n1)], axis=1)
    t0 = time.perf_counter()
    oracle.render(lf, eye, pixels=pix, threads=1)
    t1 = time.perf_counter() - t0
    return {"value": total_pix / total_t / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d random pixels of one %dx%d eye of the same workload (each call also builds the "
                      "per-view meshes it needs), %.1f s" % (total_pix, eye.width, eye.height, total_t),
            "single_thread": {"value": n1 / t1 / 1e6, "unit": UNIT, "cores": 1,
                              "sample": "%d random pixels, %.1f s" % (n1, t1)}}


def quality_vs_oracle(r, lf, head, n_pixels):
    """Max-abs and PSNR of this storage form against the FP64 oracle on random
    pixels of both eyes of one head pose (RGB, peak 1, pixels valid on both)."""
    import numpy as np
    import torch

    import oracle

    rng = np.random.default_rng(3)
    out = r.render(head)
    torch.cuda.synchronize()
    diffs, mism = [], 0
    n_rec = n_rec_diff = 0
    for eye, img in zip(head, out):
        pix = np.stack([rng.integers(0, eye.width, n_pixels), rng.integers(0, eye.height, n_pixels)], axis=1)
        ref = oracle.render(lf, eye, pixels=pix)["rgba"]
        g = img.cpu().numpy().astype(np.float64)[pix[:, 1], pix[:, 0]]
        valid = (ref[:, 3] > 0) & (g[:, 3] > 0)
        mism += int(np.sum((ref[:, 3] > 0) != (g[:, 3] > 0)))
        diffs.append(g[valid][:, :3] - ref[valid][:, :3])
        # coverage records at the same pixels against the FP64-decision oracle (the definition)
        got = r.render_inspect(eye, max_records=32)
        ref64 = oracle.render(lf, eye, pixels=pix, fragments=True, max_slots=32, decisions="fp64")
        want = {}
        for f in ref64["frags"]:
            i, j = pix[int(f["pixel"])]
            want[(int(j) * eye.width + int(i), int(f["view"]))] = (
                int(f["n_cover"]), int(f["winner"]), int(f["min_id"]), int(f["max_id"]), int(f["id_hash"]))
        have = {}
        for i, j in pix:
            k = int(j) * eye.width + int(i)
            for rec in got["records"][k][:min(int(got["counts"][k]), 32)]:
                have[(k, int(rec["view"]))] = (int(rec["n_cover"]), int(rec["winner"]), int(rec["min_id"]),
                                               int(rec["max_id"]), int(rec["id_hash"]))
        keys = set(want) | set(have)
        n_rec += len(keys)
        n_rec_diff += sum(1 for k in keys if want.get(k) != have.get(k))
        del got
    d = np.concatenate(diffs)
    mse = float(np.mean(d * d)) if d.size else 0.0
    # reconstruction error of the method itself: every valid pixel of both eyes
    # against the analytic ray-cast image of the scene (RGBA8, view-independent shading)
    import scene

    sq, n_truth = 0.0, 0
    for eye, img in zip(head, out):
        g = img.cpu().numpy().astype(np.float64)
        t = scene.truth_image(lf, eye).astype(np.float64) / 255.0
        valid = g[..., 3] > 0
        e = g[valid][:, :3] - t[valid][:, :3]
        sq += float(np.sum(e * e))
        n_truth += e.size
    mse_t = sq / n_truth if n_truth else 0.0
    return {"vs": "FP64 oracle", "pixels": int(d.shape[0]), "max_abs": float(np.abs(d).max()) if d.size else 0.0,
            "records_vs_fp64_decisions": {"compared": n_rec, "differ": n_rec_diff,
                                          "frac": n_rec_diff / n_rec if n_rec else 0.0,
                                          "what": "(pixel, view) coverage records of the sampled pixels against "
                                                  "the oracle taking its snap, depth and disk decisions in FP64"},
            "psnr_db": (10.0 * math.log10(1.0 / mse)) if mse > 0 else float("inf"), "valid_mask_mismatches": mism,
            "psnr_vs_analytic_truth_db": (10.0 * math.log10(1.0 / mse_t)) if mse_t > 0 else float("inf"),
            "truth": "analytic ray cast of the scene, every valid pixel of both eyes"}


def workload_config(args, desc: str, n_heads: int, world: int) -> dict:
    """The `config` of the default workload's line, the same in both arms."""
    return {"workload": desc, "texture_storage": args.tex, "mesh_storage": args.mesh, "tile": args.tile,
            "disks": args.disk, "head_poses": n_heads,
            "l2": "flushed (256 MiB write) between steps, outside the timed events",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    lf, heads, desc = make_workload(args.workload, max(args.poses, 1), 0)
    import numpy as np

    import oracle

    cores = os.cpu_count() or 1
    rng = np.random.default_rng(11)
    # a step is the oracle on a bounded random sample of both eyes of one head pose:
    # large enough that each call's mesh building (about 0.2 s per eye at rig scale)
    # is a small part of it, as in the measured arm's cpu_baseline; a long --steps
    # run stops once this much CPU time is spent, after at least 3 timed steps
    per_step = 200000
    budget_s = 150.0
    times, pixels = [], 0
    t_start = time.perf_counter()
    for s in range(args.warmup + args.steps):
        if len(times) >= 3 and time.perf_counter() - t_start > budget_s:
            break
        head = heads[s % len(heads)]
        t0 = time.perf_counter()
        for eye in head:
            pix = np.stack([rng.integers(0, eye.width, per_step // 2), rng.integers(0, eye.height, per_step // 2)],
                           axis=1)
            oracle.render(lf, eye, pixels=pix, threads=cores)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            pixels += per_step
    total = sum(times)
    value = pixels / total / 1e6
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": len(times), "steps_requested": args.steps, "warmup": args.warmup,
           "ms_per_step": 1000 * total / len(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(args, desc, len(heads), world),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "%d random pixels per step over both eyes of one head pose (each oracle "
                                      "call also builds the meshes of the views it selects), %d steps, %.1f s"
                                      % (per_step, len(times), total)},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def make_batch(rank: int):
    """The tiny scene and cap rig, 64 head poses x stereo = 128 eyes whose sizes are
    drawn per pose from {512^2, 1024^2, 1440x1600, 2048^2} (90 degrees horizontal)."""
    import scene

    lf = scene.tiny_light_field(1)
    rng = scene.SplitMix64(4242 + 104729 * rank)
    sizes = [(512, 512), (1024, 1024), (1440, 1600), (2048, 2048)]
    eyes = []
    for _ in range(64):
        w, h = sizes[int(rng.uniform(0, 4)) % 4]
        eyes += scene.head_pose_eyes(rng, w, h, 90.0, yaw_range=(-math.radians(10), math.radians(10)),
                                     pitch_deg=10.0)
    desc = ("batched: tiny cap rig (16 views 128^2, 32^2 meshes), 64 head poses x stereo = 128 eyes of "
            "mixed sizes {512^2, 1024^2, 1440x1600, 2048^2}, one persistent launch per step replayed "
            "as a CUDA graph, tile shape and grid autotuned")
    return lf, eyes, desc


def run_batch(args):
    import torch

    rank, world, local = dist_env()
    init_dist(world)
    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_08860_gb300 as lfm

    lf, eyes, desc = make_batch(rank)
    r = lfm.Renderer(local, max_eyes=len(eyes))
    r.load_views(lf, tex_format=args.tex)
    r.build_meshes(lf, mesh_format=args.mesh)
    stream = torch.cuda.current_stream()
    outs = [torch.empty((e.height, e.width, 4), dtype=torch.float32, device="cuda") for e in eyes]
    px = sum(e.width * e.height for e in eyes)
    # the same eyes through lf_render one eye at a time with the default
    # configuration, for comparison (one warm-up pass, then one timed pass)
    for e, o in zip(eyes, outs):
        r.render([e], out=[o])
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for e, o in zip(eyes, outs):
        r.render([e], out=[o])
    b.record(stream)
    b.synchronize()
    plain_ms = a.elapsed_time(b)
    tune = r.tune_batch(eyes, out=outs, replays=2)
    uniq = r.unique_texels(eyes, lf.width, lf.height)
    for _ in range(args.warmup):
        r.render_batch(eyes, out=outs)
    torch.cuda.synchronize()
    barrier_all()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        r.render_batch(eyes, out=outs)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    assert r.stats()["error_word"] == 0
    # the raster kernel's own duration, from a timing context (eager launches of
    # the same persistent sequence with the tuned tile shape and grid)
    rt = lfm.Renderer(local, tile=tune["tile"], max_eyes=len(eyes), timing=True)
    rt.load_views(lf, tex_format=args.tex)
    rt.build_meshes(lf, mesh_format=args.mesh)
    raster_ms = []
    for k in range(max(3, args.steps // 2)):
        flush.zero_()
        rt.render_batch(eyes, out=outs)
        st = rt.stats()
        if k >= 1:
            raster_ms.append(st["ms_raster"])
    rt.close()
    total_ms = max_over_ranks(sum(x.elapsed_time(y) for x, y in ev))
    value = whole_job_rate(px * args.steps, total_ms, world)
    # end to end through lf_render_host (batch form): all eyes delivered to
    # pinned host memory, two frames in flight, each with its own host images
    need = 2 * px * 16
    avail = host_memory_available()
    e2e = {"value": None, "unit": UNIT, "h2d_bytes_per_step": 160 * len(eyes), "d2h_bytes_per_step": px * 16}
    if avail >= 4 * need:
        e2e["value"], e2e["frame_latency_ms"] = host_e2e(r, [eyes], [o.shape for o in outs], flush, stream,
                                                         max(3, args.steps // 4), px, world, form="batch",
                                                         in_flight=2)
        e2e["what"] = E2E_WHAT % ("lf_render_host (batch)", "all %d eye images" % len(eyes))
    else:
        e2e["skipped"] = "host memory: %.1f GB available, %.1f GB of pinned images needed (x4 margin)" % (
            avail / 1e9, need / 1e9)
    peak, peak_kind = measured_peak()
    tex_bytes = {"f32": 16, "u8": 4, "bf16": 8, "fp8": 4}[args.tex]
    raster_bytes = uniq * tex_bytes + px * 16
    mean_raster = statistics.mean(raster_ms)
    achieved = raster_bytes / (mean_raster / 1000.0) / 1e9
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "texture_storage": args.tex, "mesh_storage": args.mesh,
                   "eyes": len(eyes), "pixels_per_step": px,
                   "l2": "flushed (256 MiB write) between steps, outside the timed events"},
        "autotune": {"tile": list(tune["tile"]), "blocks_per_sm": tune["blocks_per_sm"], "ms": tune["ms"],
                     "tried": [{"tile": list(t["tile"]), "blocks_per_sm": t["blocks_per_sm"], "ms": t["ms"]}
                               for t in tune["tried"]]},
        "plain_per_eye_calls": {"ms_per_step": plain_ms, "value": px / (plain_ms / 1000.0) / 1e6, "unit": UNIT},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": ncu_traffic("raster_batch128_%s_persistent" % args.tex),
                     "kernel": "raster_kernel (persistent)",
                     "peak_source": peak_kind + " (HBM copy)", "algorithmic_bytes_per_launch": raster_bytes,
                     "unique_texels_per_step": uniq, "ms_per_launch": mean_raster},
        "e2e": e2e,
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(result), flush=True)
    r.close()
    finish_dist(world)
    return 0


REFINE_FLOP_PER_PX = 2 * (27 * 32 + 288 * 32 + 288 * 3)  # 21,888: the three convolutions' multiply-adds x 2
# A training step per pixel: the forward pass, dL/d(input) of layers 3 and 2 (layer 1's is not needed),
# and the three layers' weight gradients, as multiply-adds x 2 (63,936).
TRAIN_FLOP_PER_PX = 2 * ((27 * 32 + 288 * 32 + 288 * 3) + (27 * 32 + 288 * 32) + (27 * 32 + 288 * 32 + 288 * 3))
TRAIN_LAUNCHES_PER_STEP = 13  # count, 3 convolutions, 3 weight gradients, 2 backward convolutions, 3 reductions, Adam, pack


def measured_tensor_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def _supersampled(r, eye, s):
    """Render at s x s samples per pixel and box-filter RGB weighted by alpha."""
    import numpy as np
    import scene
    import torch

    big = scene.Eye(eye.pose, np.asarray(eye.intr, dtype=np.float64) * s, eye.width * s, eye.height * s)
    img = r.render([big])[0]
    pool = lambda t: torch.nn.functional.avg_pool2d(t.permute(2, 0, 1)[None], s)[0].permute(1, 2, 0)
    rgb, a = pool(img[..., :3] * img[..., 3:4]), pool(img[..., 3:4])
    out = torch.zeros((eye.height, eye.width, 4), device=img.device)
    ok = a[..., 0] > 0
    out[..., :3] = torch.where(ok[..., None], rgb / a.clamp_min(1e-12), torch.zeros_like(rgb))
    out[..., 3] = ok.float()
    return out.contiguous()


def _psnr(a, b):
    import torch

    v = (a[..., 3] > 0) & (b[..., 3] > 0)
    d = (a[..., :3] - b[..., :3])[v].double()
    return float(10.0 * torch.log10(1.0 / (d * d).mean()))


def run_refine(args):
    """The refinement alone: lf_refine of a stereo pair of 1440x1600 RGBA images
    (smooth synthetic colour fields with 2 % holes) with seeded weights."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    init_dist(world)
    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_08860_gb300 as lfm

    rng = np.random.default_rng(5 + rank)
    yy, xx = np.mgrid[0:1600, 0:1440].astype(np.float32)
    imgs = np.zeros((2, 1600, 1440, 4), np.float32)
    for k in range(2):
        for c in range(3):
            imgs[k, ..., c] = 0.5 + 0.3 * np.sin(rng.uniform(0.01, 0.2) * xx + rng.uniform(0.01, 0.2) * yy)
        imgs[k, ..., 3] = (rng.uniform(size=(1600, 1440)) > 0.02).astype(np.float32)
    imgs[..., :3] *= imgs[..., 3:4]
    x = torch.from_numpy(imgs).cuda()
    y = torch.empty_like(x)
    r = lfm.Renderer(local)
    r.load_refiner(lfm.init_refiner_params(3, out_scale=0.3))
    r.set_refine_kernel(args.refine_kernel)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        r.refine(x, out=y)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        r.refine(x, out=y)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    # end to end: the pair from pinned host memory, lf_refine, the result back
    # to pinned host memory, one step at a time (events around all three)
    hx = x.cpu().pin_memory()
    hy = torch.empty(hx.shape, dtype=torch.float32, pin_memory=True)
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(max(3, args.steps // 4))]
    for a, b in e2e_ev:
        flush.zero_()
        a.record(stream)
        x.copy_(hx, non_blocking=True)
        r.refine(x, out=y)
        hy.copy_(y, non_blocking=True)
        b.record(stream)
    torch.cuda.synchronize()
    r.get_refiner()
    ms = [a.elapsed_time(b) for a, b in ev]
    px = 2 * 1440 * 1600
    mean = max_over_ranks(sum(ms)) / len(ms)
    e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in e2e_ev)) / len(e2e_ev)
    peak, peak_kind = measured_tensor_peak()
    achieved = REFINE_FLOP_PER_PX * px / (mean / 1000.0) / 1e12
    result = {
        "metric": METRIC, "value": whole_job_rate(px, mean, world), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "refinement only: lf_refine of 2 x 1440x1600 RGBA images (one launch), seeded "
                               "weights", "refine_kernel": args.refine_kernel,
                   "l2": "flushed (256 MiB write) between steps, outside the timed events"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": ncu_traffic(REFINE_PROFILE, REFINE_SOURCES) if args.refine_kernel == "fused" else None,
                     "kernel": "refine_fused_kernel" if args.refine_kernel == "fused" else "conv_tc_kernel x3",
                     "peak_source": peak_kind + " bf16 (burst)", "flop_per_pixel": REFINE_FLOP_PER_PX},
        "e2e": {"value": whole_job_rate(px, e2e_ms, world), "unit": UNIT, "h2d_bytes_per_step": px * 16,
                "d2h_bytes_per_step": px * 16,
                "what": "the pair copied from pinned host memory, lf_refine, the result copied back to pinned "
                        "host memory; events around all three, one step at a time"},
        "gpu_launches": (1 if args.refine_kernel == "fused" else 3) * args.steps,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(result), flush=True)
    r.close()
    finish_dist(world)
    return 0


def run_train(args):
    """One training step of the refinement (lf_refine_train_step: forward, loss,
    backward, weight gradients, Adam) on a batch of 16 synthetic 256^2 crops and
    targets (smooth colour fields, 2 % holes; the target a perturbed copy), the
    batch shape of the learned workload's training."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    init_dist(world)
    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_08860_gb300 as lfm

    n, h, w = 16, 256, 256
    rng = np.random.default_rng(7 + rank)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float32)
    imgs = np.zeros((n, h, w, 4), np.float32)
    for k in range(n):
        for c in range(3):
            imgs[k, ..., c] = 0.5 + 0.3 * np.sin(rng.uniform(0.02, 0.3) * xx + rng.uniform(0.02, 0.3) * yy)
        imgs[k, ..., 3] = (rng.uniform(size=(h, w)) > 0.02).astype(np.float32)
    imgs[..., :3] *= imgs[..., 3:4]
    tgt = imgs.copy()
    tgt[..., :3] = np.clip(tgt[..., :3] * 0.9 + 0.05 * np.sin(0.05 * xx)[None, ..., None], 0, 1) * tgt[..., 3:4]
    x = torch.from_numpy(imgs).cuda()
    t = torch.from_numpy(tgt).cuda()
    r = lfm.Renderer(local)
    r.load_refiner(lfm.init_refiner_params(3, out_scale=0.1))
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        r.refine_train_step(x, t, 1e-3)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        r.refine_train_step(x, t, 1e-3)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    # end to end: the batch from pinned host memory, the step, the refiner state
    # (weights, gradient, moments, step, loss) read back by lf_get_refiner
    hx, ht = x.cpu().pin_memory(), t.cpu().pin_memory()
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(max(3, args.steps // 4))]
    for a, b in e2e_ev:
        flush.zero_()
        a.record(stream)
        x.copy_(hx, non_blocking=True)
        t.copy_(ht, non_blocking=True)
        r.refine_train_step(x, t, 1e-3)
        st = r.get_refiner()
        b.record(stream)
    torch.cuda.synchronize()
    assert np.isfinite(st["loss"])
    ms = [a.elapsed_time(b) for a, b in ev]
    px = n * h * w
    mean = max_over_ranks(sum(ms)) / len(ms)
    e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in e2e_ev)) / len(e2e_ev)
    peak, peak_kind = measured_tensor_peak()
    achieved = TRAIN_FLOP_PER_PX * px / (mean / 1000.0) / 1e12
    result = {
        "metric": "training pixels/s of the learned refinement (Mpix/s), % of the BF16 tensor roofline",
        "value": whole_job_rate(px, mean, world), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "refinement training step: batch of 16 RGBA crops 256x256 with targets, "
                               "forward, loss, backward, weight gradients, Adam",
                   "l2": "flushed (256 MiB write) between steps, outside the timed events"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "conv_tc_kernel x5 + wgrad_tc_kernel x3 (one step)",
                     "peak_source": peak_kind + " bf16 (burst)", "flop_per_pixel": TRAIN_FLOP_PER_PX},
        "e2e": {"value": whole_job_rate(px, e2e_ms, world), "unit": UNIT, "h2d_bytes_per_step": 2 * px * 16,
                "d2h_bytes_per_step": 4 * 4 * 11011 + 8,
                "what": "the batch and targets copied from pinned host memory, one training step, the refiner "
                        "state read back (lf_get_refiner); events around all of it, one step at a time"},
        "gpu_launches": TRAIN_LAUNCHES_PER_STEP * args.steps,
        "clocks": clk,
        "loss": float(st["loss"]),
    }
    if rank == 0:
        print(json.dumps(result), flush=True)
    r.close()
    finish_dist(world)
    return 0


PREFILTER_VIEWS_PER_STEP = 8


def pick_prefilter_samples(lfm, J: int):
    """The first seed whose stratified sample set's weights rho sigma sum to more
    than 0.6 of their absolute sum (a set whose Lanczos lobes do not nearly cancel)."""
    import numpy as np

    for seed in range(1000):
        S = lfm.prefilter_samples(J, seed).astype(np.float64)
        w = (1.0 - np.sqrt(S[:, 0])) * np.sinc(S[:, 2]) * np.sinc(S[:, 2] / 2) * np.sinc(S[:, 3]) * np.sinc(S[:, 3] / 2)
        if w.sum() > 0.6 * np.abs(w).sum():
            return S.astype(np.float32), seed, float(w.sum() / np.abs(w).sum())
    raise RuntimeError("no balanced prefilter sample set")


def run_prefilter(args):
    """The light field prefilter (Sec. 5, Eq. 5) at rig scale: images of the
    1,024-view real-time model replaced by Monte Carlo estimates over each
    view's disk and a Lanczos-2 pixel basis, with Lbar rendered by the method
    from a 4,096-view dense model with 256^2 meshes.  Timed: blocks of 8 views
    per step.  Quality: stereo eyes rendered from the prefiltered and from the
    original images, each against the analytic ray-cast truth."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    init_dist(world)
    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_08860_gb300 as lfm
    import scene

    t0 = time.perf_counter()
    lf = scene.rig_light_field(1, n_heads=2)
    dense = scene.build_light_field(lf.prims, scene.fibonacci_directions(args.dense_views), lf.width, lf.height,
                                    120.0, args.dense_grid)
    gen_s = time.perf_counter() - t0
    J = args.samples
    samples, seed, balance = pick_prefilter_samples(lfm, J)
    rt = lfm.Renderer(local)
    rt.load_views(lf)
    rt.build_meshes(lf)
    rd = lfm.Renderer(local, max_eyes=J, tri_capacity=J << 20, timing=True)
    rd.load_views(dense, tex_format="u8")
    rd.build_meshes(dense)
    V, W, H = PREFILTER_VIEWS_PER_STEP, lf.width, lf.height
    n_blocks = lf.n_views // V
    out = torch.empty((V, H, W, 4), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    first = lambda k: ((k + rank) % n_blocks) * V  # noqa: E731  ranks take different blocks
    S = args.supersample
    for k in range(args.warmup):
        rt.prefilter(rd, samples, first_view=first(k), n_views=V, supersample=S, out=out)
    torch.cuda.synchronize()
    barrier_all()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    raster_ms = []
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        rt.prefilter(rd, samples, first_view=first(args.warmup + k), n_views=V, supersample=S, out=out)
        ev[k][1].record(stream)
        raster_ms.append(rd.stats()["ms_raster"])  # the last view's batched dense render
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev))
    texels = V * W * H
    value = whole_job_rate(texels * args.steps, total_ms, world)
    # end to end: the prefiltered block copied to pinned host memory each step
    host = torch.empty(out.shape, dtype=torch.float32, pin_memory=True)
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(max(3, args.steps // 2))]
    for k, (a, b) in enumerate(e2e_ev):
        flush.zero_()
        a.record(stream)
        rt.prefilter(rd, samples, first_view=first(k), n_views=V, supersample=S, out=out)
        host.copy_(out, non_blocking=True)
        b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in e2e_ev)) / len(e2e_ev)

    # roofline of the dense raster: the J renders of one view read these texels and write J images
    P, K, (Ws, Hs) = rt.prefilter_cameras(0, samples, supersample=S)
    cams = [scene.Eye(P[j], K[j], Ws, Hs) for j in range(J)]
    uniq = rd.unique_texels(cams, dense.width, dense.height)
    raster_bytes = uniq * 4 + J * Ws * Hs * 16
    mean_raster = statistics.mean(raster_ms)
    peak, peak_kind = measured_peak()
    achieved = raster_bytes / (mean_raster / 1000.0) / 1e9
    result = {
        "metric": "prefiltered source texels/s (Sec. 5, Eq. 5)", "value": value, "unit": "Mtexel/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "prefilter: rig model (1,024 Fibonacci views 1024^2 at 120 deg, 64^2 meshes), "
                               "Lbar from a %d-view dense model with %d^2 meshes (u8 textures); %d samples per "
                               "pixel (stratified, seed %d, weight balance %.2f); %d views per step; renders "
                               "at %dx" % (args.dense_views, args.dense_grid, J, seed, balance, V, S),
                   "l2": "flushed (256 MiB write) between steps, outside the timed events",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "per_step": {"renders": V * J, "render_pixels": V * J * Ws * Hs, "ms_per_render": total_ms / args.steps / (V * J)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "raster_kernel (persistent): the %d dense renders of one view" % J,
                     "peak_source": peak_kind + " (HBM copy)", "algorithmic_bytes_per_launch": raster_bytes,
                     "unique_texels_per_launch": uniq, "ms_per_launch": mean_raster},
        "e2e": {"value": whole_job_rate(texels, e2e_ms, world), "unit": "Mtexel/s", "h2d_bytes_per_step": 16 * J,
                "d2h_bytes_per_step": texels * 16,
                "what": "lf_prefilter from host samples plus the prefiltered block copied to pinned host memory"},
        "gpu_launches": 4 * V * args.steps,
        "clocks": clk,
        "scene_generation_s": gen_s,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["quality"] = prefilter_quality(lfm, scene, rt, rd, lf, samples, local, S)
        from oracle import prefilter as opf

        rng = np.random.default_rng(13)
        pix = np.stack([rng.integers(0, W, 200), rng.integers(0, H, 200)], axis=1)
        t1 = time.perf_counter()
        opf.prefilter(lf, dense, 0, samples.astype(np.float64), pixels=pix, sparse=True, threads=os.cpu_count())
        dt = time.perf_counter() - t1
        result["cpu_baseline"] = {"value": 200 / dt / 1e6, "unit": "Mtexel/s", "cores": os.cpu_count() or 1,
                                  "kind": "oracle", "sample": "200 random texels of view 0, %d samples, renders "
                                                              "evaluated only where read, %.1f s" % (J, dt)}
    if rank == 0:
        print(json.dumps(result), flush=True)
    rt.close()
    rd.close()
    finish_dist(world)
    return 0


def prefilter_quality(lfm, scene, rt, rd, lf, samples, local, supersample=1):
    """PSNR against the analytic truth of the rig's stereo eyes rendered from the
    original images and from images prefiltered (every view the eyes select)."""
    import dataclasses

    import numpy as np

    active = np.zeros(lf.n_views, dtype=bool)
    for e in lf.eyes:
        active |= np.asarray(rt.render_inspect(e, max_records=1)["active"]).astype(bool)
    ids = np.nonzero(active)[0]
    images = lf.images.copy()
    t0 = time.perf_counter()
    runs = np.split(ids, np.nonzero(np.diff(ids) != 1)[0] + 1)
    for run in runs:
        for c0 in range(0, len(run), 32):
            part = run[c0:c0 + 32]
            o = rt.prefilter(rd, samples, first_view=int(part[0]), n_views=len(part),
                             supersample=supersample).cpu().numpy()
            rgb8 = np.clip(np.rint(o[..., :3] * 255.0), 0, 255).astype(np.uint8)
            for m, v in enumerate(part):
                ok = o[m, ..., 3] > 0
                images[v][ok, :3] = rgb8[m][ok]
    pre_s = time.perf_counter() - t0
    rp = lfm.Renderer(local)
    lfp = dataclasses.replace(lf, images=images)
    rp.load_views(lfp)
    rp.build_meshes(lfp)
    res = {}
    for name, r in (("original", rt), ("prefiltered", rp)):
        sq, n = 0.0, 0
        for e in lf.eyes:
            img = r.render([e])[0].cpu().numpy().astype(np.float64)
            t = scene.truth_image(lf, e)[..., :3].astype(np.float64) / 255.0
            ok = img[..., 3] > 0
            d = img[ok][:, :3] - t[ok]
            sq += float(np.sum(d * d))
            n += d.size
        res["psnr_%s_db" % name] = 10.0 * math.log10(1.0 / (sq / n))
    rp.close()
    res.update({"vs": "analytic ray-cast truth, every valid pixel of %d eyes (1440x1600)" % len(lf.eyes),
                "views_prefiltered": int(len(ids)), "prefilter_s": pre_s,
                "gain_db": res["psnr_prefiltered_db"] - res["psnr_original_db"]})
    return res


def run_learned(args):
    """Learned refinement: train y = x + f(x) on pairs the method generates (the
    fast light field's render of a 256x256 crop vs a 2x2-supersampled render
    of a denser light field of the same scene), evaluate on held-out
    1440x1600 eyes against the dense render, and time the refined stereo
    render (lf_render_refined, fused tcgen05 refinement) against the plain one."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    init_dist(world)
    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_08860_gb300 as lfm
    import scene

    t0 = time.time()
    prims = scene.sphere_scene(1, 8)
    fast = scene.build_light_field(prims, scene.fibonacci_directions(1024), 1024, 1024, 120.0, 64)
    dense = scene.build_light_field(prims, scene.fibonacci_directions(args.dense_views), 1024, 1024, 120.0,
                                    args.dense_grid)
    gen_s = time.time() - t0
    rf = lfm.Renderer(local, max_eyes=2)
    rf.load_views(fast)
    rf.build_meshes(fast)
    rd = lfm.Renderer(local, max_eyes=1, tri_capacity=96 << 20)
    rd.load_views(dense, tex_format="u8")
    rd.build_meshes(dense)
    rng = scene.SplitMix64(5151 + 104729 * rank)

    def crop(size=256):
        e = scene.head_pose_eyes(rng, 1440, 1600, 100.0)[int(rng.uniform(0.0, 2.0)) % 2]
        ox, oy = int(rng.uniform(0, 1440 - size)), int(rng.uniform(0, 1600 - size))
        K = np.asarray(e.intr, dtype=np.float64).copy()
        K[2] -= ox
        K[3] -= oy
        return scene.Eye(e.pose, K, size, size)

    # ---- training pairs (the method on both sides)
    t0 = time.time()
    X = torch.empty((args.pairs, 256, 256, 4), device="cuda")
    T = torch.empty_like(X)
    for k in range(args.pairs):
        e = crop()
        rf.render([e], out=[X[k]])
        T[k] = _supersampled(rd, e, 2)
    torch.cuda.synchronize()
    pairs_s = time.time() - t0

    # ---- training (BF16 tensor-core forward/backward, Adam on FP32 master weights)
    rf.load_refiner(lfm.init_refiner_params(1, out_scale=0.1))
    g = torch.Generator().manual_seed(0)
    losses = []
    t0 = time.time()
    for it in range(args.train_steps):
        idx = torch.randint(0, args.pairs, (16,), generator=g)
        rf.refine_train_step(X[idx].contiguous(), T[idx].contiguous(), 2e-3 if it < 0.7 * args.train_steps else 4e-4)
        if it % 250 == 0 or it == args.train_steps - 1:
            losses.append(rf.get_refiner()["loss"])
    torch.cuda.synchronize()
    train_s = time.time() - t0
    del X, T

    # ---- held-out evaluation against the dense reference
    rf.set_refine_kernel("fused")
    eval_eyes = []
    while len(eval_eyes) < args.eval_eyes:
        eval_eyes += scene.head_pose_eyes(rng, 1440, 1600, 100.0)
    eval_eyes = eval_eyes[:args.eval_eyes]
    p_plain, p_ref = [], []
    targets = []
    for k, e in enumerate(eval_eyes):
        x = rf.render([e])[0]
        y = rf.refine(x)
        t = _supersampled(rd, e, 2)
        p_plain.append(_psnr(x, t))
        p_ref.append(_psnr(y, t))
        if k < 8:
            targets.append(t)
    forms = {"f32": float(np.mean(p_plain[:8]))}
    for fmt in ("u8", "bf16", "fp8"):
        rq = lfm.Renderer(local, max_eyes=2)
        rq.load_views(fast, tex_format=fmt)
        rq.build_meshes(fast)
        forms[fmt] = float(np.mean([_psnr(rq.render([e])[0], t) for e, t in zip(eval_eyes[:8], targets)]))
        rq.close()
    del targets
    # the dense reference itself against the FP64 oracle on sampled pixels
    dense_check = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        e = eval_eyes[0]
        prng = np.random.default_rng(17)
        # a 96x96 window: the oracle builds meshes only for the few dense views it selects
        cx0, cy0 = int(prng.integers(0, e.width - 96)), int(prng.integers(0, e.height - 96))
        pix = np.stack([cx0 + prng.integers(0, 96, 200), cy0 + prng.integers(0, 96, 200)], axis=1)
        t1 = time.time()
        ref = oracle.render(dense, e, pixels=pix, threads=os.cpu_count())["rgba"]
        got = rd.render([e])[0].cpu().numpy()[pix[:, 1], pix[:, 0]].astype(np.float64)
        v = (ref[:, 3] > 0) & (got[:, 3] > 0)
        dense_check = {"pixels": int(v.sum()), "max_abs": float(np.abs(got[v, :3] - ref[v, :3]).max()),
                       "valid_mismatches": int(np.sum((ref[:, 3] > 0) != (got[:, 3] > 0))),
                       "oracle_s": time.time() - t1}
    rd.close()

    # ---- timing: refined stereo frames vs plain ones, and the fused kernel alone
    heads = [eval_eyes[2 * k:2 * k + 2] for k in range(min(4, len(eval_eyes) // 2))]
    stream = torch.cuda.current_stream()
    outs = [torch.empty((1600, 1440, 4), device="cuda") for _ in range(2)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    px = 2 * 1440 * 1600

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            fn(k)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    for k in range(args.warmup):
        rf.render_refined(heads[k % len(heads)], out=outs)
    pair = torch.stack([rf.render([e])[0].clone() for e in heads[0]])
    refined = torch.empty_like(pair)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms_refined = timed(lambda k: rf.render_refined(heads[k % len(heads)], out=outs), args.steps)
    clk = clocks.stop()
    ms_plain = timed(lambda k: rf.render(heads[k % len(heads)], out=outs), args.steps)
    ms_kernel = timed(lambda k: rf.refine(pair, out=refined), max(20, args.steps // 4))
    # end to end: host poses in, both refined images delivered to pinned host memory
    e2e_value, e2e_latency = host_e2e(rf, heads, [o.shape for o in outs], flush, stream,
                                      max(20, args.steps // 4), px, world, form="refined")
    st = rf.get_refiner()  # raises if the fused kernel reported a failed wait
    if args.save_refiner and rank == 0:
        # the trained weights, with the held-out quality they scored, for the default line's learned form
        meta = {"vs": "dense reference (method, %d views, %d^2 meshes, 2x2 supersampled)" % (
                    args.dense_views, args.dense_grid),
                "eval_eyes": len(eval_eyes), "eye": "1440x1600, 100 deg",
                "psnr_plain_db": float(np.mean(p_plain)), "psnr_refined_db": float(np.mean(p_ref)),
                "gain_db": float(np.mean(p_ref) - np.mean(p_plain)),
                "training": {"pairs": args.pairs, "crop": 256, "steps": args.train_steps, "batch": 16,
                             "scene": "8 spheres (seed 1), fast light field 1024 Fibonacci views 1024^2 at 120 deg, "
                                      "64^2 meshes"},
                "written_by": "python bench.py --workload learned --save-refiner <path>"}
        np.savez(args.save_refiner, params=st["params"].astype(np.float32), meta=json.dumps(meta))
    total = max_over_ranks(sum(ms_refined))
    value = whole_job_rate(px * args.steps, total, world)
    kern = statistics.mean(ms_kernel)
    peak, peak_kind = measured_tensor_peak()
    achieved = REFINE_FLOP_PER_PX * px / (kern / 1000.0) / 1e12
    cores = os.cpu_count() or 1
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "learned refinement: 8 spheres, fast light field 1024 Fibonacci views 1024x1024 "
                               "(120 deg), 64x64 meshes; dense reference %d views, %dx%d meshes, 2x2 "
                               "supersampled; stereo 2x1440x1600 refined eyes" % (
                                   args.dense_views, args.dense_grid, args.dense_grid),
                   "refine_kernel": "fused tcgen05 (one launch per stereo pair)",
                   "l2": "flushed (256 MiB write) between steps, outside the timed events"},
        "plain_render": {"ms_per_step": statistics.mean(ms_plain),
                         "value": px / (statistics.mean(ms_plain) / 1000.0) / 1e6, "unit": UNIT},
        "refine_kernel": {"ms_per_launch_2_eyes": kern, "value": px / (kern / 1000.0) / 1e6, "unit": UNIT},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": ncu_traffic(REFINE_PROFILE, REFINE_SOURCES),
                     "kernel": "refine_fused_kernel",
                     "peak_source": peak_kind + " bf16 (burst)", "flop_per_pixel": REFINE_FLOP_PER_PX,
                     "algorithmic_flop_per_launch": REFINE_FLOP_PER_PX * px},
        "quality": {"vs": "dense reference (method, %d views, %d^2 meshes, 2x2 supersampled)" % (
                        args.dense_views, args.dense_grid),
                    "eval_eyes": len(eval_eyes), "psnr_plain_db": float(np.mean(p_plain)),
                    "psnr_refined_db": float(np.mean(p_ref)),
                    "gain_db": float(np.mean(p_ref) - np.mean(p_plain)),
                    "psnr_plain_by_texture_form_db_first8": forms, "dense_reference_vs_fp64_oracle": dense_check},
        "training": {"pairs": args.pairs, "crop": 256, "steps": args.train_steps, "batch": 16,
                     "ms_per_step_wall": 1000.0 * train_s / max(1, args.train_steps), "loss_trace": losses,
                     "pairs_s": pairs_s, "scene_generation_s": gen_s, "adam_step": st["step"]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 320, "d2h_bytes_per_step": px * 16,
                "frame_latency_ms": e2e_latency, "what": E2E_WHAT % ("lf_render_host (refined)", "both refined eye images")},
        "gpu_launches": 4 * args.steps,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import refine as oref

        x = pair[0].cpu().numpy().astype(np.float64)
        pw = st["params"].astype(np.float64)
        t1 = time.perf_counter()
        oref.forward(x[:400], pw)
        dt = time.perf_counter() - t1
        result["cpu_baseline"] = {"value": 400 * 1440 / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                                  "sample": "refinement forward (numpy FP64) of a 400x1440 band of one eye, "
                                            "%.1f s; the render itself runs at the rig cpu_baseline rate" % dt}
    if rank == 0:
        print(json.dumps(result), flush=True)
    rf.close()
    finish_dist(world)
    return 0


REFINER_WEIGHTS = os.path.join(ROOT, "paper_1810_08860_gb300", "refiner_weights.npz")


def time_steps(fn, n, flush, stream):
    """CUDA-event durations (ms) of n calls of fn(k), each after an L2 flush outside the events."""
    import torch

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for k in range(n):
        flush.zero_()
        ev[k][0].record(stream)
        fn(k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def form_quality(r, lf, head, n_pixels, seed=5):
    """Max-abs and PSNR against the FP64 oracle on random pixels of one head pose,
    and PSNR against the analytic ray cast over every valid pixel."""
    import numpy as np
    import torch

    import oracle
    import scene

    rng = np.random.default_rng(seed)
    out = r.render(head)
    torch.cuda.synchronize()
    d, sq, nt = [], 0.0, 0
    for eye, img in zip(head, out):
        g = img.cpu().numpy().astype(np.float64)
        pix = np.stack([rng.integers(0, eye.width, n_pixels), rng.integers(0, eye.height, n_pixels)], axis=1)
        ref = oracle.render(lf, eye, pixels=pix)["rgba"]
        gs = g[pix[:, 1], pix[:, 0]]
        v = (ref[:, 3] > 0) & (gs[:, 3] > 0)
        d.append(gs[v, :3] - ref[v, :3])
        t = scene.truth_image(lf, eye).astype(np.float64) / 255.0
        ok = g[..., 3] > 0
        e = g[ok][:, :3] - t[ok][:, :3]
        sq += float(np.sum(e * e))
        nt += e.size
    d = np.concatenate(d)
    mse = float(np.mean(d * d)) if d.size else 0.0
    return {"max_abs_vs_fp64_oracle": float(np.abs(d).max()) if d.size else 0.0,
            "psnr_vs_fp64_oracle_db": 10.0 * math.log10(1.0 / mse) if mse > 0 else float("inf"),
            "psnr_vs_analytic_truth_db": 10.0 * math.log10(nt / sq) if sq > 0 else float("inf"),
            "oracle_pixels": int(d.shape[0])}


def forms_block(args, lfm, r, lf, heads, plain, flush, stream, local, peak, mean_u):
    """The batched, reduced-precision and learned forms, each timed on this GPU in
    this process beside the plain FP32 form (`plain`: its Mpix/s), with its own
    roofline fraction and quality."""
    import numpy as np
    import torch

    px = sum(e.width * e.height for e in heads[0])
    out_bytes = px * 16
    steps = 2 * len(heads)
    forms = {}
    # ---- precision (pattern 1): the same 8 stereo poses with u8 / BF16 / FP8 textures and FP16 meshes
    outs = [torch.empty((e.height, e.width, 4), dtype=torch.float32, device="cuda") for e in heads[0]]
    for fmt, tb in (("u8", 4), ("bf16", 8), ("fp8", 4)):
        rq = lfm.Renderer(local)
        rq.load_views(lf, tex_format=fmt)
        rq.build_meshes(lf, mesh_format="f16")
        for k in range(3):
            rq.render(heads[k % len(heads)], out=outs)
        raster = []

        def step(k):
            rq.render(heads[k % len(heads)], out=outs, stream=stream)

        ms = []
        for k in range(steps):
            ms += time_steps(lambda _: step(k), 1, flush, stream)
        # the raster kernel's own duration: the same steps with per-kernel events
        rq.set_timing(True)
        for k in range(steps):
            time_steps(lambda _: step(k), 1, flush, stream)
            raster.append(rq.stats()["ms_raster"])
        mean_ms, mean_raster = statistics.mean(ms), statistics.mean(raster)
        rbytes = mean_u * tb + out_bytes
        forms["texture_%s_mesh_f16" % fmt] = {
            "value": px / (mean_ms / 1000.0) / 1e6, "unit": UNIT, "ms_per_step": mean_ms, "steps": steps,
            "vs_plain": px / (mean_ms / 1000.0) / 1e6 / plain,
            "roofline": {"bound": "hbm", "frac": rbytes / (mean_raster / 1000.0) / 1e9 / peak,
                         "algorithmic_bytes_per_launch": rbytes, "ms_per_launch": mean_raster},
            "quality": form_quality(rq, lf, heads[0], 1000)}
        rq.close()
    # ---- batch (pattern 2): 128 eyes of mixed sizes, autotuned, one graph replay per step
    blf, beyes, bdesc = make_batch(0)
    rb = lfm.Renderer(local, max_eyes=len(beyes))
    rb.load_views(blf)
    rb.build_meshes(blf)
    bouts = [torch.empty((e.height, e.width, 4), dtype=torch.float32, device="cuda") for e in beyes]
    bpx = sum(e.width * e.height for e in beyes)
    tune = rb.tune_batch(beyes, out=bouts, replays=1)
    buniq = rb.unique_texels(beyes, blf.width, blf.height)
    for _ in range(2):
        rb.render_batch(beyes, out=bouts)
    bms = time_steps(lambda k: rb.render_batch(beyes, out=bouts), 6, flush, stream)
    assert rb.stats()["error_word"] == 0
    rt = lfm.Renderer(local, tile=tune["tile"], max_eyes=len(beyes), timing=True)
    rt.load_views(blf)
    rt.build_meshes(blf)
    braster = []
    for k in range(4):
        flush.zero_()
        rt.render_batch(beyes, out=bouts)
        if k:
            braster.append(rt.stats()["ms_raster"])
    rt.close()
    bq = {}
    rng = np.random.default_rng(9)
    dmax = 0.0
    import oracle

    for k in range(0, len(beyes), 32):  # four eyes of the batch against the oracle
        e = beyes[k]
        pix = np.stack([rng.integers(0, e.width, 500), rng.integers(0, e.height, 500)], axis=1)
        ref = oracle.render(blf, e, pixels=pix)["rgba"]
        g = bouts[k].cpu().numpy().astype(np.float64)[pix[:, 1], pix[:, 0]]
        v = (ref[:, 3] > 0) & (g[:, 3] > 0)
        bq["valid_mismatches"] = bq.get("valid_mismatches", 0) + int(np.sum((ref[:, 3] > 0) != (g[:, 3] > 0)))
        if v.any():
            dmax = max(dmax, float(np.abs(g[v, :3] - ref[v, :3]).max()))
    bq["max_abs_vs_fp64_oracle"] = dmax
    bmean, brast = statistics.mean(bms), statistics.mean(braster)
    bbytes = buniq * 16 + bpx * 16
    forms["batch_128_eyes"] = {
        "value": bpx / (bmean / 1000.0) / 1e6, "unit": UNIT, "ms_per_step": bmean, "pixels_per_step": bpx,
        "vs_plain": bpx / (bmean / 1000.0) / 1e6 / plain, "workload": bdesc,
        "autotune": {"tile": list(tune["tile"]), "blocks_per_sm": tune["blocks_per_sm"]},
        "roofline": {"bound": "hbm", "frac": bbytes / (brast / 1000.0) / 1e9 / peak,
                     "algorithmic_bytes_per_launch": bbytes, "ms_per_launch": brast},
        "quality": bq}
    rb.close()
    del bouts
    # ---- learned (pattern 4): the refined stereo render with the stored trained weights
    stored = None
    if os.path.exists(REFINER_WEIGHTS):
        z = np.load(REFINER_WEIGHTS)
        r.load_refiner(z["params"].astype(np.float32))
        stored = json.loads(str(z["meta"]))
    else:
        r.load_refiner(lfm.init_refiner_params(1, out_scale=0.1))
    r.set_refine_kernel("fused")
    for k in range(3):
        r.render_refined(heads[k % len(heads)], out=outs)
    lms = time_steps(lambda k: r.render_refined(heads[k % len(heads)], out=outs), steps, flush, stream)
    pair = torch.stack([o.clone() for o in outs])
    refined = torch.empty_like(pair)
    kms = time_steps(lambda k: r.refine(pair, out=refined), 8, flush, stream)
    r.get_refiner()  # raises if a wait of the fused kernel gave up
    tpeak, tkind = measured_tensor_peak()
    kern = statistics.mean(kms)
    lmean = statistics.mean(lms)
    forms["learned_refined"] = {
        "value": px / (lmean / 1000.0) / 1e6, "unit": UNIT, "ms_per_step": lmean, "steps": steps,
        "vs_plain": px / (lmean / 1000.0) / 1e6 / plain,
        "roofline": {"bound": "tensor", "kernel": "refine_fused_kernel", "ms_per_launch": kern,
                     "frac": REFINE_FLOP_PER_PX * px / (kern / 1000.0) / 1e12 / tpeak,
                     "peak_source": tkind + " bf16 (burst)"},
        "quality": stored if stored is not None else "no stored weights: timed with untrained weights"}
    return forms


def run_twolevel(args):
    """Two-level progressive rendering (Sec. 7.2) at rig scale: the rig light
    field is the streamed fine level (1,024 views of 1024^2, a page pool of a
    quarter of them), a 256-view light field of the same scene the resident
    coarse level.  The head turns 0.6 degrees per frame; each frame renders the
    stereo pair with what is resident, reads the fine views it selected, lets
    the host cache (FIFO) admit up to --budget of the missing ones, and copies
    those images from pinned host memory into their pages."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    init_dist(world)
    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_08860_gb300 as lfm
    import scene

    prims = scene.sphere_scene(1, 24)
    fine = scene.build_light_field(prims, scene.fibonacci_directions(1024), 1024, 1024, 120.0, 64, name="fine")
    coarse = scene.build_light_field(prims, scene.fibonacci_directions(256), 1024, 1024, 120.0, 64, name="coarse")
    import dataclasses

    both = dataclasses.replace(
        fine, poses=np.concatenate([fine.poses, coarse.poses]), intr=np.concatenate([fine.intr, coarse.intr]),
        images=np.concatenate([fine.images, coarse.images]), depth=np.concatenate([fine.depth, coarse.depth]),
        disk_c=np.concatenate([fine.disk_c, coarse.disk_c]), disk_r=np.concatenate([fine.disk_r, coarse.disk_r]),
        name="two-level")
    nf, pages = fine.n_views, args.pages
    r = lfm.Renderer(local)
    r.load_views(both)
    r.build_meshes(both)
    r.set_levels(nf, pages)
    host = torch.from_numpy(fine.images).pin_memory().numpy()  # the streamed images, pinned
    cache = lfm.PageCache(nf, pages)
    rng = scene.SplitMix64(8191 + 104729 * rank)
    centre = rng.in_ball(0.2)
    yaw0 = rng.uniform(0.0, 2 * math.pi)
    K = scene.intrinsics_for_fov(1440, 1600, 100.0)

    def head(f):
        R = scene.look_rotation(scene.yaw_pitch_dir(yaw0 + math.radians(0.6) * f, 0.0))
        right = R[:, 0]
        return [scene.Eye(scene.pose_array(R, centre - 0.032 * right), K, 1440, 1600),
                scene.Eye(scene.pose_array(R, centre + 0.032 * right), K, 1440, 1600)]

    outs = [torch.empty((1600, 1440, 4), dtype=torch.float32, device="cuda") for _ in range(2)]
    px = 2 * 1440 * 1600
    stream = torch.cuda.current_stream()
    rec = []
    clocks = ClockSampler(local)
    for f in range(args.warmup + args.steps):
        if f == args.warmup:
            torch.cuda.synchronize()
            barrier_all()
            clocks.start()
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r.render(head(f), out=outs, stream=stream)
        e1.record(stream)
        wanted = r.levels_wanted()  # waits for the frame
        st = r.stats()
        miss = int((cache.pages()[wanted] < 0).sum()) if len(wanted) else 0
        adm = cache.frame(wanted, args.budget)
        if adm:
            r.upload_pages([v for v, _ in adm], [p for _, p in adm], [host[v] for v, _ in adm], stream=stream)
        t1 = time.perf_counter()
        if f >= args.warmup:
            rec.append({"render_ms": e0.elapsed_time(e1), "frame_ms": 1000 * (t1 - t0), "wanted": int(len(wanted)),
                        "missing": miss, "admitted": len(adm), "drawn": sum(st["active_views"])})
    clk = clocks.stop()
    # the raster kernel's own duration: frames of the last head pose with per-kernel events
    # (timed frames above run without them, as a user's calls do)
    r.set_timing(True)
    raster_ms = []
    for _ in range(5):
        r.render(head(args.warmup + args.steps - 1), out=outs, stream=stream)
        raster_ms.append(r.stats()["ms_raster"])
    r.set_timing(False)
    render_ms = max_over_ranks(sum(x["render_ms"] for x in rec)) / len(rec)
    frame_ms = max_over_ranks(sum(x["frame_ms"] for x in rec)) / len(rec)
    # quality of the last frame against the analytic truth, beside the fine level alone
    last = head(args.warmup + args.steps - 1)
    prog = [o.cpu().numpy().astype(np.float64) for o in r.render(last, out=outs)]
    rf = lfm.Renderer(local)
    rf.load_views(fine)
    rf.build_meshes(fine)
    full = [o.cpu().numpy().astype(np.float64) for o in rf.render(last)]
    rf.close()

    def psnr(imgs):
        sq, n = 0.0, 0
        for e, g in zip(last, imgs):
            t = scene.truth_image(fine, e).astype(np.float64) / 255.0
            v = g[..., 3] > 0
            d = g[v][:, :3] - t[v][:, :3]
            sq += float(np.sum(d * d))
            n += d.size
        return 10.0 * math.log10(n / sq) if sq > 0 else float("inf")

    valid = [float((g[..., 3] > 0).mean()) for g in prog]
    result = {
        "metric": METRIC, "value": whole_job_rate(px, render_ms, world), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": render_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "two-level progressive (Sec. 7.2): fine level 1024 Fibonacci views 1024^2 (120 deg), "
                               "64^2 meshes, streamed into %d device pages; coarse level 256 views, resident; "
                               "24 spheres; stereo 2x1440x1600 eyes, head turning 0.6 deg per frame" % pages,
                   "pages": pages, "budget_per_frame": args.budget, "texture_storage": "f32"},
        "loop": {"value": whole_job_rate(px, frame_ms, world), "unit": UNIT, "ms_per_frame": frame_ms,
                 "what": "render + wanted views read back + cache decision + page uploads from pinned host memory"},
        "frames": {"mean_wanted": statistics.mean(x["wanted"] for x in rec),
                   "mean_missing": statistics.mean(x["missing"] for x in rec),
                   "mean_admitted": statistics.mean(x["admitted"] for x in rec),
                   "mean_drawn_views": statistics.mean(x["drawn"] for x in rec),
                   "raster_ms": statistics.mean(raster_ms),
                   "upload_bytes_per_frame": 1024 * 1024 * 4 * statistics.mean(x["admitted"] for x in rec)},
        "quality": {"psnr_vs_analytic_truth_db": psnr(prog), "fine_level_alone_db": psnr(full),
                    "valid_fraction": valid},
        "e2e": {"value": None, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "note": "see loop (the streamed images are this workload's host traffic)"},
        "gpu_launches": 6 * args.steps,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(result), flush=True)
    cache.close()
    r.close()
    finish_dist(world)
    return 0


def issue_roofline(args, ms_launch, clk, raster_bytes, hbm_peak, px):
    """The raster against the SM instruction-issue roofline: the warp instructions
    per launch of the committed full-section capture (while its source hash
    matches) over this run's launch time, against 4 issue slots per SM per clock
    at the sampled SM clock - the bound that keeps the kernel below its HBM
    roofline."""
    import torch

    prof = "raster_%s_%s_%s" % (args.workload, args.tex, args.tile)
    inst = ncu_value(prof, "warp_instructions_per_launch")
    if inst is None or args.disk != "round" or args.workload != "rig":
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    peak = sms * 4 * mhz * 1e6
    floor_s = inst / peak
    return {"bound": "issue", "unit": "warp inst/s", "achieved": inst / (ms_launch / 1000.0), "peak": peak,
            "frac": inst / (ms_launch / 1000.0) / peak, "warp_inst_per_launch": inst, "warp_inst_per_pixel": inst / px,
            "issue_active_pct_ncu": ncu_value(prof, "issue_active_pct"),
            "hbm_frac_at_issue_peak": raster_bytes / floor_s / 1e9 / hbm_peak,
            "source": "profiles/%s.txt (instructions of a rig256 capture of the same eyes and meshes)" % prof}


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    init_dist(world)
    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_08860_gb300 as lfm

    tw, th = (int(x) for x in args.tile.split("x"))
    lf, heads, desc = make_workload(args.workload, max(args.poses, 1), rank)
    if args.disk == "oval":  # Sec. 4.4: extents reach the farthest Delaunay 1-ring neighbour per axis
        import dataclasses

        from paper_1810_08860_gb300 import disks

        lf = dataclasses.replace(lf, disk_ext=disks.oval_extents(lf))
    r = lfm.Renderer(local, tile=(tw, th))
    r.load_views(lf, tex_format=args.tex)
    r.build_meshes(lf, mesh_format=args.mesh)
    stream = torch.cuda.current_stream()
    outs = [torch.empty((e.height, e.width, 4), dtype=torch.float32, device="cuda") for e in heads[0]]
    px_per_step = sum(e.width * e.height for e in heads[0])
    out_bytes = px_per_step * 16
    tex_bytes = {"f32": 16, "u8": 4, "bf16": 8, "fp8": 4}[args.tex]
    vtx_bytes = 4 if args.mesh == "f32" else 2

    # Algorithmic bytes: distinct texels each stereo frame reads, plus its output.
    uniq = [r.unique_texels(h, lf.width, lf.height) for h in heads]
    active = []
    for h in heads:
        r.render(h, out=outs)
        active.append(sum(r.stats()["active_views"]))
    mean_u = statistics.mean(uniq)
    mesh_bytes = statistics.mean(active) * lf.grid_n ** 2 * vtx_bytes  # depth grids of the active views

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]

    def step(k, timed_pair=None):
        head = heads[k % len(heads)]
        flush.zero_()
        if timed_pair:
            timed_pair[0].record(stream)
        r.render(head, out=outs, stream=stream)
        if timed_pair:
            timed_pair[1].record(stream)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    barrier_all()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    for k in range(args.steps):
        step(args.warmup + k, ev[k])
        assert r.stats()["error_word"] == 0  # waits for the step
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms))
    barrier_all()
    value = whole_job_rate(px_per_step * args.steps, total_ms, world)

    # Each kernel's own duration: the same steps again with the library's
    # per-kernel events on the launch stream (which rule out the programmatic
    # launches of the timed steps above, so they are kept out of those).
    r.set_timing(True)
    raster_ms, setup_v_ms, setup_t_ms = [], [], []
    for k in range(min(args.steps, 500)):
        step(args.warmup + k)
        st = r.stats()
        raster_ms.append(st["ms_raster"])
        setup_v_ms.append(st["ms_view_setup"])
        setup_t_ms.append(st["ms_tri_setup"])
        assert st["error_word"] == 0
    r.set_timing(False)

    # End to end through lf_render_host: host poses in, both images delivered to
    # pinned host memory (the copy of one frame overlaps the render of the next).
    e2e_value, e2e_latency = host_e2e(r, heads, [o.shape for o in outs], flush, stream,
                                      max(3, args.steps // 2), px_per_step, world)

    peak, peak_kind = measured_peak()
    mean_raster = statistics.mean(raster_ms)
    raster_bytes = mean_u * tex_bytes + out_bytes
    achieved = raster_bytes / (mean_raster / 1000.0) / 1e9
    step_bytes = raster_bytes + mesh_bytes
    step_achieved = step_bytes / (total_ms / args.steps / 1000.0) / 1e9
    traffic = ncu_traffic("raster_%s%s_%s_%s" % (args.workload, "_oval" if args.disk == "oval" else "", args.tex,
                                                  args.tile))
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args, desc, len(heads), world),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": "raster_kernel", "peak_source": peak_kind + " (HBM copy)",
                     "algorithmic_bytes_per_launch": raster_bytes,
                     "unique_texels_per_step": mean_u, "ms_per_launch": mean_raster},
        "step_roofline": {"bytes_per_step": step_bytes, "achieved": step_achieved, "frac": step_achieved / peak,
                          "unit": "GB/s"},
        "issue_roofline": issue_roofline(args, mean_raster, clk, raster_bytes, peak, px_per_step),
        "phases_ms": {"view_setup": statistics.mean(setup_v_ms), "tri_setup": statistics.mean(setup_t_ms),
                      "raster": mean_raster},
        "active_views_per_step": statistics.mean(active),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 160 * len(heads[0]),
                "d2h_bytes_per_step": out_bytes, "frame_latency_ms": e2e_latency,
                "what": E2E_WHAT % ("lf_render_host", "both eye images")},
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
    }
    # the CPU-baseline leg (the only part of this arm that runs the oracle) also compares
    # sampled pixels of the GPU frame against it
    if rank == 0 and not args.no_cpu_baseline and args.quality_pixels > 0:
        result["quality"] = quality_vs_oracle(r, lf, heads[0], args.quality_pixels)
    # the other forms of the method beside this plain one (their quality checks also run the oracle)
    if rank == 0 and not args.no_cpu_baseline and not args.no_forms and args.workload == "rig" and \
            args.tex == "f32" and args.disk == "round":
        result["forms"] = forms_block(args, lfm, r, lf, heads, value / world, flush, stream, local, peak, mean_u)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(lf, heads[0][0], args.cpu_seconds)
    if rank == 0:
        print(json.dumps(result), flush=True)
    r.close()
    finish_dist(world)
    return 0


def main():
    args = parse_args()
    if args.steps is None:
        args.steps = 20 if args.impl == "reference" else {"rig": 2000, "batch": 60, "learned": 1000,
                                                          "refine": 1000, "prefilter": 10, "twolevel": 120}.get(args.workload, 400)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "prefilter":
        return run_prefilter(args)
    if args.workload == "refine":
        return run_refine(args)
    if args.workload == "train":
        return run_train(args)
    if args.workload == "twolevel":
        return run_twolevel(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
