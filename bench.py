#!/usr/bin/env python3
"""Benchmark of live sparse TSDF fusion on the room-scale workload.

Workload: ground plane + 50 seeded spheres/boxes in a 3 m room, 640x480 depth
maps (fx = fy = 525) along a 300-frame seeded spline, noise sigma = 1.5e-3 z^2
plus 2 % edge dropout, fused into a 2048^3 grid of 1.5 mm voxels (truncation
7.5 mm, pool of 2^20 8^3-voxel blocks), float32 T and P.

One step = one pass of the whole hot path over the sequence: reset the volume,
then for each frame allocate -> integrate (Alg. 3) -> raycast at the frame's
pose. ``value`` is frames fused per second over all ranks (each rank fuses its
own replica: weak scaling), inputs resident in HBM. ``e2e`` is the same through
the public Python API with each depth map copied from pinned host memory and
the last raycast maps read back every step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the CPU oracle (plain FP64 C++, all host cores) on a
bounded sample of the same workload (each step: one whole frame fused and
raycast, all timed) and prints the same JSON line with "impl": "reference".
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "room-scale plain FP32: 640x480, 2048^3 grid of 1.5 mm voxels, 300 frames"
METRIC, UNIT = "frames/s", "frames/s"
def launches_per_frame(graph: bool, persistent: bool) -> int:
    """Kernels per frame: allocation 5 (mark, count, assign, commit, chi fill)
    and integration 3 (depth tiles, cull, integrate); the raycast's raster and
    march, plus the ray order before a persistent march, plus its own range
    clear and range cull unless a graph step's integrate cull did both."""
    return 5 + 3 + 2 + (1 if persistent else 0) + (0 if graph else 2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=300)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other configurations the default line carries (batched K=8, capsules in three "
                         "storage formats, FP16 + batched + learned against plain FP32)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--launch-shape", default=None, metavar="VPT,CTAS,PERSISTENT",
                    help="room workload: set the launch shape (integrate voxels per thread, integrate CTAs per SM, "
                         "1 for the persistent raycast) instead of autotuning it")
    ap.add_argument("--block-capacity", type=int, default=None, help="pool size in blocks")
    ap.add_argument("--mode", choices=["graph", "direct"], default="graph",
                    help="graph: each step one CUDA graph launch; direct: one C-ABI call per stage")
    ap.add_argument("--storage", choices=["f32", "f16", "snorm16"], default="f32",
                    help="storage of T for --workload capsules")
    ap.add_argument("--oracle-sample", type=int, default=0,
                    help="capsules: compare this many sampled voxels with the FP64 oracle (per-voxel replay)")
    ap.add_argument("--icp-iterations", type=int, default=6, help="tracking: ICP iterations per frame")
    ap.add_argument("--workload", choices=["room", "batched", "capsules", "sphere", "tracking", "mesh", "shift",
                                                "combined"],
                    default="room",
                    help="room: per-frame live fusion (2048^3, 1.5 mm); batched: 3000^3 grid of 1 mm voxels, "
                         "1000 frames fused K=8 per graph launch, raycast per batch; capsules: 1280x1024 "
                         "small objects on a 4096^3 grid of 0.15 mm voxels; sphere: the 160x120 parity scene; "
                         "tracking: raycast -> ICP -> fuse at the registered pose; mesh: marching-cubes extraction")
    ap.add_argument("--cpu-frames", type=int, default=3, help="oracle sample: whole frames fused and raycast")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(seconds: float, world: int, device="cpu") -> float:
    """The slowest rank's time: every rank gets the all-reduce MAX of its own."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput of weak-scaled replicas: all ranks' units over the
    slowest rank's time."""
    return units_per_rank * world / seconds_max


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# CPU oracle sample (the reported CPU baseline and the reference arm)
# ----------------------------------------------------------------------------

def oracle_sample(seq, frames, ov=None, start=0):
    """Time the oracle on ``frames`` whole frames of the sequence from ``start``:
    each fuses the frame (allocate + Alg. 3 over every allocated block) and
    raycasts every pixel at the frame's pose, as one step of the GPU path does.
    Nothing is extrapolated: returns (measured seconds per frame, seconds of
    fusion, seconds of raycasting, the oracle volume)."""
    import oracle
    if ov is None:
        ov = oracle.OracleVolume(seq.volume, seq.intr)
    t_fuse = t_ray = 0.0
    for k in range(start, start + frames):
        f = k % seq.n_frames
        t0 = time.perf_counter()
        ov.fuse(seq.depth[f], seq.poses[f])
        t1 = time.perf_counter()
        ov.raycast(seq.poses[f])
        t2 = time.perf_counter()
        t_fuse += t1 - t0
        t_ray += t2 - t1
    return (t_fuse + t_ray) / frames, t_fuse, t_ray, ov


def make_sequence(n_frames, device, block_capacity=None, workload="room"):
    from paper_1311_7194_b300 import synth
    if workload == "batched":
        return synth.room_sequence(seed=1, n_frames=n_frames, device=device, grid_dim=3000, voxel_size=1e-3,
                                   block_capacity=block_capacity or (1 << 21), origin=(0.0, -0.036, 0.0))
    return synth.room_sequence(seed=1, n_frames=n_frames, device=device, block_capacity=block_capacity or (1 << 20))


def room_config(seq, world, n_frames):
    """The workload's config, identical in both arms (the GPU launch details go
    to the line's "launch" key)."""
    H, W = seq.intr.height, seq.intr.width
    return {"workload": WORKLOAD, "width": W, "height": H, "grid_dim": int(seq.volume.grid_dim),
            "voxel_size_m": float(seq.volume.voxel_size), "truncation_m": float(seq.volume.truncation),
            "block_capacity": int(seq.volume.block_capacity), "sequence_frames": n_frames,
            "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2: 368 MB of depth maps and a 4 GB block pool per step"}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    frames_per_step = 1
    seq = make_sequence(max(1, min(args.frames, (args.warmup + args.steps) * frames_per_step)), "cpu")
    ov = None
    k = 0
    for _ in range(args.warmup):
        *_, ov = oracle_sample(seq, frames_per_step, ov, start=k)
        k += frames_per_step
    per, fuse, ray = [], 0.0, 0.0
    for _ in range(args.steps):
        t, tf, tr, ov = oracle_sample(seq, frames_per_step, ov, start=k)
        k += frames_per_step
        per.append(t)
        fuse += tf
        ray += tr
    sec = sum(per) / len(per)
    value = 1.0 / sec
    cores = oracle.num_threads()
    H, W = seq.intr.height, seq.intr.width
    sample = (f"each step: the oracle fuses one whole {W}x{H} frame (allocate + Alg. 3 over every allocated "
              f"block, FP64) and raycasts every pixel at its pose, all timed; frames {args.warmup}..{k - 1} of "
              f"the sequence after {args.warmup} warm-up frames")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sec, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": room_config(seq, world, args.frames), "frames_per_step": frames_per_step,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "fuse_s_per_frame": fuse / args.steps, "raycast_s_per_frame": ray / args.steps,
                             "rays_per_s": H * W * args.steps / ray},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def _sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


# DRAM traffic of a stage measured by ncu on this workload
# (dram__bytes_read.sum + dram__bytes_write.sum over the stage's kernels), per
# voxel update for the integrate stage and per traced unique byte for the
# raycast stage,
# with the hash of the kernel source it was measured on; a value is dropped
# when that source changes.
NCU_TRAFFIC = {
    # frames 100-109, 10 launches each of depth_tiles + cull (which also makes
    # the raycast's visible list) + integrate: 2185.1 MB over 76.55 M voxel updates.
    # "same_kernels": later sources whose changes lie only in kernels this
    # workload does not launch (7cae83e0...: depth_tiles_mlp_kernel, which runs
    # only with a variance network set, reads its depths from a shared patch)
    "integrate": {"sha": "970d6d56551aa5a6", "same_kernels": ["7cae83e001bdf50c"], "bytes_per_unit": 28.55},
    # same frames, 10 launches each of raster + ray order + persistent raycast:
    # 1015.7 MB against 783.8 MB of traced unique bytes, i.e. DRAM bytes per
    # algorithmic byte
    "raycast": {"sha": "e3bf95a41e672e86", "bytes_per_unit": 1.2959},
}
STAGE_SOURCES = {"integrate": "tsdf_integrate.cu", "raycast": "tsdf_raycast.cu"}
TRACE_EVERY = 10


def ncu_traffic(stage, units):
    rec = NCU_TRAFFIC.get(stage)
    src = os.path.join(ROOT, "paper_1311_7194_b300", "csrc", STAGE_SOURCES[stage])
    if not rec or _sha(src) not in (rec.get("sha"), *rec.get("same_kernels", ())):
        return None
    return rec["bytes_per_unit"] * units


# L2 throughput of the persistent raycast kernel as a fraction of its peak (ncu
# "L2 Cache Throughput", one capture of the room workload), with the hash of the
# kernel source it was measured on; dropped when that source changes.
NCU_L2 = {"raycast": {"sha": "e3bf95a41e672e86", "frac": 0.133}}


def ncu_l2_frac(stage):
    rec = NCU_L2.get(stage)
    src = os.path.join(ROOT, "paper_1311_7194_b300", "csrc", STAGE_SOURCES[stage])
    if not rec or rec.get("sha") != _sha(src):
        return None
    return rec["frac"]


def raycast_latency_model(steps_per_ray, rays, sec, sm_mhz, ctas_per_sm=8, threads=128):
    """The raycast as a latency-bound loop: every ray is a chain of dependent
    samples (steps_per_ray, traced), each a block-table load followed by its
    voxel loads. With every resident lane (ctas_per_sm x threads per SM, the
    persistent kernel's launch bounds) busy, a lane spends
    sec x clock x lanes / (rays x steps) cycles per step: the figure to set
    against two dependent L2-hit latencies, the cost of one step when a lane
    never waits for its warp."""
    import torch
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    lanes = n_sm * ctas_per_sm * threads
    mhz = sm_mhz or 2032.0
    cycles = sec * mhz * 1e6 * lanes / (rays * steps_per_ray)
    return {"dependent_steps_per_ray": steps_per_ray, "rays": rays, "resident_lanes": lanes,
            "cycles_per_step_per_lane": cycles, "sm_mhz": mhz}


def choose_launch(vol, args, depth_dev, seq, n_tune=20):
    """The launch shape of a workload's volume: the one --launch-shape names,
    else the autotuner's pick on the first frames (it empties the volume;
    results do not depend on the shape), else the library's default."""
    if getattr(args, "launch_shape", None):
        vpt, ctas, persistent = (int(x) for x in args.launch_shape.split(","))
        vol.set_launch_config(integrate_voxels_per_thread=vpt, integrate_ctas_per_sm=ctas,
                              raycast_persistent=persistent)
        return vol.launch_config()
    if not getattr(args, "no_autotune", False):
        n = min(n_tune, int(depth_dev.shape[0]))
        tuned, _ = vol.autotune([depth_dev[k] for k in range(n)], seq.intr, seq.poses[:n],
                                os.environ.get("TSDF_AUTOTUNE_CACHE"))
        return tuned
    return vol.launch_config()


def raycast_algorithmic_bytes(counts, n_blocks, H, W, own_cull=True):
    """Unique bytes one raycast must move: the distinct 32-byte sectors of T
    and of the block table its samples read, the block list read by the range
    cull (16 B per block, when the raycast makes its own visible list; a graph
    step makes it in the integrate cull's pass), the near / far range tiles
    (8 B per 4x4 pixels) and the depth, normal and vertex maps written (28 B
    per pixel)."""
    tiles = ((W + 3) // 4) * ((H + 3) // 4)
    return (32.0 * (counts["t_sectors"] + counts["table_sectors"]) + (16.0 * n_blocks if own_cull else 0.0)
            + 8.0 * tiles + 28.0 * H * W)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1311_7194_b300 import build as pkg_build
    from paper_1311_7194_b300 import tsdf
    from paper_1311_7194_b300.pipeline import FusionPipeline

    rank, local_rank, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if rank == 0:
        pkg_build.build()
    if world > 1:
        dist.barrier()
    tsdf.load()

    seq = make_sequence(args.frames, dev, args.block_capacity)
    F, H, W = seq.depth.shape
    depth_dev = torch.from_numpy(seq.depth).to(dev)
    vol = tsdf.Volume.from_params(seq.volume)
    tuned = choose_launch(vol, args, depth_dev, seq)
    pipe = FusionPipeline(vol, seq.intr, dev, graph=args.mode == "graph")
    stream = torch.cuda.current_stream()

    def step(stage_events=None):
        vol.reset()
        for k in range(F):
            if stage_events is None:
                pipe.step(depth_dev[k], seq.poses[k])
            elif pipe.graph is not None:
                pipe.graph.set_events(stage_events[k])     # recorded as nodes of the step's graph
                pipe.step(depth_dev[k], seq.poses[k])
            else:
                e = stage_events[k]
                e[0].record(stream)
                vol.allocate(depth_dev[k], seq.intr, seq.poses[k])
                e[1].record(stream)
                vol.integrate(depth_dev[k], seq.intr, seq.poses[k])
                e[2].record(stream)
                vol.raycast(seq.intr, seq.poses[k], out=pipe.maps)
                e[3].record(stream)
        if pipe.graph is not None:
            pipe.graph.set_events(None)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    vol.check()

    # timed region: whole steps bracketed by barrier + synchronize
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    elapsed = t0.elapsed_time(t1) / 1000.0
    st = vol.stats()
    vol.check()
    # Stage times (the rooflines' launch durations): the same steps timed again
    # with event nodes at the stage boundaries of every frame. They sit between
    # the stages' kernels, so they cut the programmatic-launch overlap there;
    # the headline region above carries none.
    ev = [[[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(F)] for _ in range(args.steps)]
    for s in range(args.steps):
        step(ev[s])
    torch.cuda.synchronize()
    clk = clocks.stop()
    stage = np.zeros(3)
    for s in range(args.steps):
        for k in range(F):
            e = ev[s][k]
            stage += [e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])]
    stage_ms_per_step = stage / args.steps

    elapsed_max = max_over_ranks(elapsed, world, dev)
    frames_total = F * args.steps * world
    value = job_throughput(F * args.steps, world, elapsed_max)
    updates_per_step = st["voxel_updates_total"]
    rays_per_step = F * H * W

    # per-frame work counts (one extra, untimed step, synchronising per frame);
    # every TRACE_EVERY-th frame's raycast is traced for its unique bytes
    vol.reset()
    n_blocks, visible, updates, rc_bytes, rc_steps = [], [], [], [], []
    for k in range(F):
        vol.allocate(depth_dev[k], seq.intr, seq.poses[k])
        vol.integrate(depth_dev[k], seq.intr, seq.poses[k])
        s_ = vol.stats()
        n_blocks.append(s_["n_blocks"]); visible.append(s_["visible_blocks"]); updates.append(s_["voxel_updates"])
        if k % TRACE_EVERY == 0:
            c = vol.raycast_trace(seq.intr, seq.poses[k])
            rc_bytes.append(raycast_algorithmic_bytes(c, s_["n_blocks"], H, W, own_cull=args.mode != "graph"))
            # dependent samples along a ray: the march (jumps included), re-scans,
            # the refinement, and one round for the six independent normal samples
            rc_steps.append((c["march_samples"] + c["rescan_samples"] + c["refine_samples"]) / c["rays"] + 1.0)
    n_blocks, visible, updates = map(np.asarray, (n_blocks, visible, updates))
    peak, peak_kind = peaks()
    # integrate stage, algorithmic bytes per frame: read+write T and P of every
    # updated voxel (16 B), the depth map (4 B/px), the block list read by the
    # cull (16 B/block) and the visible list written and read (32 B each way)
    integ_bytes = 16.0 * updates + 4.0 * H * W + 16.0 * n_blocks + 64.0 * visible
    integ_sec = stage_ms_per_step[1] / 1000.0
    achieved = integ_bytes.sum() / integ_sec / 1e9
    roofline_integrate = {"kernel": "integrate stage (depth tiles + cull + Alg. 3 integrate), per frame",
                          "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                          "frac": achieved / peak, "peak_kind": peak_kind,
                          "traffic": ncu_traffic("integrate", float(updates.mean())),
                          "algorithmic_bytes_per_launch": float(integ_bytes.mean()),
                          "avg_launch_ms": 1000.0 * integ_sec / F}
    # raycast stage (the dominant one): unique bytes it must read and write
    rc_mean = float(np.mean(rc_bytes))
    rc_sec = stage_ms_per_step[2] / 1000.0 / F
    roofline = {"kernel": "raycast stage (range cull + raster + persistent march / refine / normal), per frame",
                "bound": "hbm", "achieved": rc_mean / rc_sec / 1e9, "peak": peak, "unit": "GB/s",
                "frac": rc_mean / rc_sec / 1e9 / peak, "peak_kind": peak_kind,
                "traffic": ncu_traffic("raycast", rc_mean), "algorithmic_bytes_per_launch": rc_mean,
                "avg_launch_ms": 1000.0 * rc_sec,
                "algorithmic_bytes": "distinct 32 B sectors of T and of the block table read (traced every "
                                     f"{TRACE_EVERY}th frame) + 8 B per 4x4-pixel range tile + 28 B per pixel of "
                                     "maps written (+ 16 B per allocated block for the range cull when the raycast "
                                     "makes its own visible list; a graph step makes it in the integrate cull)",
                "limiter": "instruction issue and dependent-load latency, not bandwidth: DRAM and L2 run far below "
                           "their peaks while the kernel runs (l2_frac_ncu), and the latency model below shows the "
                           "cycles each dependent step costs a lane",
                "l2_frac_ncu": ncu_l2_frac("raycast"),
                "latency_model": raycast_latency_model(float(np.mean(rc_steps)), rays_per_step / F, rc_sec,
                                                       clk.get("sm_mhz"))}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: seeded analytic room scene, quadratic depth noise, edge dropout",
            "config": room_config(seq, world, args.frames), "frames_per_step": F,
            "launch": {"mode": "one CUDA graph per frame" if args.mode == "graph" else "one C-ABI call per stage",
                       "shape": tuned or vol.launch_config(),
                       "stage_timing": "stage_ms_per_step and the rooflines' durations: a second timed pass of the "
                                       "same steps with CUDA event nodes at every stage boundary"},
            "voxel_updates_per_s": updates_per_step * args.steps * world / elapsed_max,
            "rays_per_s": rays_per_step * args.steps * world / elapsed_max,
            # the same counts over their own stage's time (stage-timing pass)
            "voxel_updates_per_s_integrate_stage": updates_per_step / (stage_ms_per_step[1] / 1000.0),
            "rays_per_s_raycast_stage": rays_per_step / (stage_ms_per_step[2] / 1000.0),
            "stage_ms_per_step": {"allocate": stage_ms_per_step[0], "integrate": stage_ms_per_step[1],
                                  "raycast": stage_ms_per_step[2]},
            "work_per_step": {"voxel_updates": int(updates_per_step), "blocks": int(st["n_blocks"]),
                              "visible_blocks": int(st["visible_blocks_total"]),
                              "rays_hit": int(st["rays_hit_total"])},
            "roofline": roofline, "roofline_integrate": roofline_integrate,
            "gpu_launches": launches_per_frame(args.mode == "graph", bool(vol.launch_config()["raycast_persistent"]))
                            * F * args.steps,
            "clocks": clk}

    # end to end through the public API with host buffers
    if not args.no_e2e:
        host = torch.from_numpy(seq.depth).pin_memory()
        out_host = [torch.empty(m.shape, dtype=torch.float32).pin_memory() for m in pipe.maps]
        for _ in range(1):
            vol.reset()
            for k in range(F):
                pipe.step_host(host[k], seq.poses[k])
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        w0 = time.perf_counter()
        for _ in range(args.steps):
            vol.reset()
            for k in range(F):
                pipe.step_host(host[k], seq.poses[k])
            for o, m in zip(out_host, pipe.maps):
                o.copy_(m, non_blocking=True)
            vol.stats()     # synchronises and reads the step's counters
        torch.cuda.synchronize()
        e2e_sec = time.perf_counter() - w0
        line["e2e"] = {"value": job_throughput(F * args.steps, world, max_over_ranks(e2e_sec, world, dev)),
                       "unit": UNIT,
                       "h2d_bytes_per_step": int(F * H * W * 4),
                       "d2h_bytes_per_step": int(28 * H * W + 11 * 8)}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        sec, tf, tr, _ = oracle_sample(seq, args.cpu_frames)
        line["cpu_baseline"] = {"value": 1.0 / sec, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": f"the oracle fuses the first {args.cpu_frames} whole frames at {W}x{H} "
                                          f"(allocate + Alg. 3 over every allocated block, FP64) and raycasts every "
                                          f"pixel of each at its pose; measured, nothing extrapolated",
                                "fuse_s_per_frame": tf / args.cpu_frames, "raycast_s_per_frame": tr / args.cpu_frames,
                                "rays_per_s": H * W * args.cpu_frames / tr}
    vol.close()
    if rank == 0 and world == 1 and not args.no_extras:
        line.update(run_extras(args))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_extras(args):
    """The other configurations, each run after the room line with 3 warm-up
    and 2 timed steps (CUDA events, inputs resident): the batched + graphed
    workload (3000^3 grid of 1 mm voxels, 1000 frames, K = 8) with its integrate
    roofline; the capsules (1280x1024, 4096^3 grid of 0.15 mm voxels, 200
    frames) with T in FP32, FP16 and snorm16 and each one's error against the
    FP64 oracle on 999 sampled voxels; and the FP16 + K = 8 + learned-variance
    form against plain FP32 on the room sequence at a stated surface-error
    bound."""
    out = {}

    def sub_args(**kw):
        a = argparse.Namespace(**vars(args))
        a.__dict__.update(dict(steps=2, warmup=3, block_capacity=None, no_autotune=args.no_autotune), **kw)
        return a

    def keep(d, keys):
        return {k: d[k] for k in keys if k in d}

    try:
        b = run_batched(sub_args(frames=1000), emit=False)
        out["batched_k8"] = keep(b, ["value", "unit", "ms_per_step", "config", "voxel_updates_per_s", "rays_per_s",
                                     "work_per_step", "roofline_integrate_batch", "launch", "clocks"])
    except Exception as e:          # the room line stands on its own
        out["batched_k8"] = {"error": repr(e)}
    caps = {}
    for storage in ("f32", "f16", "snorm16"):
        try:
            c = run_capsules(sub_args(frames=200, workload="capsules", storage=storage, oracle_sample=999),
                             emit=False)
            caps[storage] = keep(c, ["value", "unit", "ms_per_step", "voxel_updates_per_s", "rays_per_s", "dtype",
                                     "pool_bytes_per_voxel", "error_vs_fp64_oracle", "launch", "clocks"])
        except Exception as e:
            caps[storage] = {"error": repr(e)}
    out["capsules"] = {"config": "capsules: 1280x1024, 4096^3 grid of 0.15 mm voxels, 200 frames, one graph per "
                                 "frame", **caps}
    try:
        c = run_combined(sub_args(frames=300), emit=False)
        out["vs_plain_fp32"] = {"config": c["config"], "forms": c["forms"], "speedup_vs_plain": c["speedup_vs_plain"],
                                "surface_error_bound": c["surface_error_bound"], "clocks": c["clocks"]}
    except Exception as e:
        out["vs_plain_fp32"] = {"error": repr(e)}
    return out


def run_batched(args, emit=True):
    """The batched + graphed workload: 3000^3 grid of 1 mm voxels, 640x480,
    frames fused K = 8 per graph launch (tsdf_integrate_batch semantics) with a
    raycast at each batch's last pose. The integrate stage's roofline: its
    algorithmic bytes per launch are 16 B (T and P read and written once) per
    voxel that any of the K frames updates, the K depth maps (4 B per pixel),
    the block list read by the cull (16 B per block) and K visible-list entries
    written and read per visible block (64 B each), over the stage's CUDA-event
    duration in a second timed pass."""
    import numpy as np
    import torch

    from paper_1311_7194_b300 import build as pkg_build
    from paper_1311_7194_b300 import tsdf

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    pkg_build.build()
    K = 8
    n = (args.frames if args.frames != 300 else 1000) // K * K
    seq = make_sequence(n, dev, args.block_capacity, workload="batched")
    F, H, W = seq.depth.shape
    depth_dev = torch.from_numpy(seq.depth).to(dev)
    vol = tsdf.Volume.from_params(seq.volume)
    shape = choose_launch(vol, args, depth_dev, seq)
    g = tsdf.Graph(vol, seq.intr, K)
    maps = (torch.empty((H, W), device=dev), torch.empty((H, W, 3), device=dev), torch.empty((H, W, 3), device=dev))

    def step():
        vol.reset()
        for k in range(0, F, K):
            g.launch([depth_dev[k + j] for j in range(K)], seq.poses[k:k + K], maps)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    vol.check()
    clocks = ClockSampler(0)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        step()
    t1.record()
    torch.cuda.synchronize()
    sec = t0.elapsed_time(t1) / 1000.0
    st = vol.stats()
    vol.check()
    # stage times: the same steps again with event nodes at the stage boundaries
    ev = [[[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(F // K)] for _ in range(args.steps)]
    for s in range(args.steps):
        vol.reset()
        for b, k in enumerate(range(0, F, K)):
            g.set_events(ev[s][b])
            g.launch([depth_dev[k + j] for j in range(K)], seq.poses[k:k + K], maps)
        g.set_events(None)
    torch.cuda.synchronize()
    clk = clocks.stop()
    integ_ms = sum(ev[s][b][1].elapsed_time(ev[s][b][2]) for s in range(args.steps) for b in range(F // K)) / args.steps
    peak, peak_kind = peaks()
    launches = F // K
    touched, nblk = st["voxels_touched_total"], st["n_blocks"]
    # algorithmic bytes per step, with each launch's own pool size and visible
    # count (one more untimed step, read back after every launch)
    integ_bytes = 0.0
    vol.reset()
    for k in range(0, F, K):
        g.launch([depth_dev[k + j] for j in range(K)], seq.poses[k:k + K], maps)
        s_ = vol.stats()
        integ_bytes += K * 4.0 * H * W + 16.0 * s_["n_blocks"] + 64.0 * K * s_["visible_blocks"]
    integ_bytes += 16.0 * touched
    achieved = integ_bytes / (integ_ms / 1000.0) / 1e9
    line = {"metric": METRIC, "value": F * args.steps / sec, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched + graphed: 640x480, 3000^3 grid of 1 mm voxels, {F} frames, K={K} per "
                                   "graph launch, raycast per batch", "frames_per_step": F},
            "voxel_updates_per_s": st["voxel_updates_total"] * args.steps / sec,
            "rays_per_s": (F // K) * H * W * args.steps / sec,
            "work_per_step": {"voxel_updates": int(st["voxel_updates_total"]), "voxels_touched": int(touched),
                              "blocks": int(nblk)},
            "roofline_integrate_batch": {"kernel": f"integrate stage of a K={K} launch (K depth tiles + batched cull "
                                                   "+ batched Alg. 3 integrate)", "bound": "hbm",
                                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                                         "peak_kind": peak_kind, "traffic": None,
                                         "algorithmic_bytes_per_launch": integ_bytes / launches,
                                         "avg_launch_ms": integ_ms / launches},
            "launch": {"shape": shape}, "graph_instantiations": g.instantiations, "clocks": clk}
    g.close()
    vol.close()
    if emit:
        print(json.dumps(line), flush=True)
    return line


_CAPSULE_ORACLE = {}


def capsule_oracle_reference(seq, n_sample):
    """Sampled voxels of the capsule sequence replayed by the FP64 oracle (the
    same for every storage format, so computed once): block allocation over the
    whole sequence, n_sample voxels drawn from the allocated blocks, and their T
    after every frame from their block's allocation frame on."""
    import numpy as np
    import oracle
    key = (seq.depth.shape, n_sample)
    if key not in _CAPSULE_ORACLE:
        oracle.build()
        ov = oracle.OracleVolume(seq.volume, seq.intr, store_values=False)
        for k in range(seq.depth.shape[0]):
            ov.allocate(seq.depth[k], seq.poses[k], k)
        oe = ov.export(values=False)
        rng = np.random.default_rng(11)
        pick = rng.choice(oe.coords.shape[0], size=min(n_sample, oe.coords.shape[0]), replace=False)
        local = rng.integers(0, 512, size=pick.size)
        vox = oe.coords[pick] * 8 + np.stack([local & 7, (local >> 3) & 7, local >> 6], -1)
        T, P, amb = oracle.replay_voxels(seq.volume, seq.intr, list(seq.depth), seq.poses, vox,
                                         oe.alloc_frame[pick], amb_px=5e-4)
        _CAPSULE_ORACLE[key] = (oe.coords[pick], local, T, amb)
    return _CAPSULE_ORACLE[key]


def run_capsules(args, emit=True):
    """Small scenes, one graph launch per frame, T stored as float32, FP16 or
    snorm16 (P float32); optionally the error of sampled voxels against the
    FP64 oracle. capsules: high-resolution small object, 1280x1024, 4096^3 grid
    of 0.15 mm voxels, 200 frames; sphere: the tiny parity scene, 160x120,
    256^3 grid of 1 mm voxels, 10 frames."""
    import numpy as np
    import torch

    from paper_1311_7194_b300 import build as pkg_build
    from paper_1311_7194_b300 import synth, tsdf
    from paper_1311_7194_b300.pipeline import FusionPipeline

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    pkg_build.build()
    storage = {"f32": tsdf.STORAGE_F32, "f16": tsdf.STORAGE_F16, "snorm16": tsdf.STORAGE_SNORM16}[args.storage]
    if args.workload == "sphere":
        n = args.frames if args.frames != 300 else 10
        seq = synth.sphere_sequence(n_frames=n, device=dev)
        name = f"tiny sphere: 160x120, 256^3 grid of 1 mm voxels, {n} frames"
    else:
        n = args.frames if args.frames != 300 else 200
        seq = synth.capsule_sequence(n_frames=n, device=dev, block_capacity=args.block_capacity or (1 << 20))
        name = f"high-res small object: 1280x1024, 4096^3 grid of 0.15 mm voxels, {n} frames"
    F, H, W = seq.depth.shape
    depth_dev = torch.from_numpy(seq.depth).to(dev)
    vol = tsdf.Volume.from_params(seq.volume, storage=storage)
    shape = choose_launch(vol, args, depth_dev, seq)
    pipe = FusionPipeline(vol, seq.intr, dev, graph=True)

    def step():
        vol.reset()
        for k in range(F):
            pipe.step(depth_dev[k], seq.poses[k])

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    vol.check()
    clocks = ClockSampler(0)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        step()
    t1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    sec = t0.elapsed_time(t1) / 1000.0
    st = vol.stats()
    bytes_per_update = 16 if storage == tsdf.STORAGE_F32 else 12
    line = {"metric": METRIC, "value": F * args.steps / sec, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {0: "f32", 1: "f16 T / f32 P", 2: "snorm16 T / f32 P"}[storage],
            "data": "synthetic",
            "config": {"workload": name, "storage": args.storage, "frames_per_step": F},
            "voxel_updates_per_s": st["voxel_updates_total"] * args.steps / sec,
            "rays_per_s": F * H * W * args.steps / sec,
            "work_per_step": {"voxel_updates": int(st["voxel_updates_total"]), "blocks": int(st["n_blocks"])},
            "pool_bytes_per_voxel": 4 + (4 if storage == tsdf.STORAGE_F32 else 2),
            "algorithmic_bytes_per_update": bytes_per_update, "launch": {"shape": shape}, "clocks": clk}
    if args.oracle_sample > 0:
        ocoords, local, T, amb = capsule_oracle_reference(seq, args.oracle_sample)
        ge = vol.export()
        nb = seq.volume.grid_dim // 8
        keys = ge.coords[:, 0].astype(np.int64) + nb * (ge.coords[:, 1] + nb * ge.coords[:, 2].astype(np.int64))
        okeys = ocoords[:, 0].astype(np.int64) + nb * (ocoords[:, 1] + nb * ocoords[:, 2].astype(np.int64))
        order = np.argsort(keys)
        slot = order[np.searchsorted(keys[order], okeys)]
        gT = ge.T[slot, local].astype(np.float64)
        m = ~np.isnan(T) & ~amb & ~np.isnan(gT)
        e = np.abs(gT[m] - T[m]) / seq.volume.truncation
        line["error_vs_fp64_oracle"] = {"voxels": int(m.sum()), "max_over_delta": float(e.max()),
                                        "rms_over_delta": float(np.sqrt((e ** 2).mean())),
                                        "chi_mismatch": int(((np.isnan(T) != np.isnan(gT)) & ~amb).sum())}
    pipe.graph.close()
    vol.close()
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_tracking(args):
    """The paper's whole per-frame loop with registration: raycast the model at
    the last estimated pose, register the frame to those maps (tsdf_icp, point-
    to-plane, args.icp_iterations iterations), allocate and integrate at the
    registered pose. Room scene at 640x480 on a 2048^3 grid of 1.5 mm voxels,
    the camera spline spread over 1200 frames (about 5 mm per frame), first 300
    frames. Wall-clock frames/s (each ICP iteration synchronises with the host,
    which holds the pose) and the tracking error against the true poses."""
    import numpy as np
    import torch

    from paper_1311_7194_b300 import build as pkg_build
    from paper_1311_7194_b300 import synth, tsdf

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    pkg_build.build()
    n = args.frames
    seq = synth.room_sequence(seed=1, n_frames=n, trajectory_frames=4 * n, device=dev,
                              block_capacity=args.block_capacity or (1 << 20))
    F, H, W = seq.depth.shape
    d = torch.from_numpy(seq.depth).to(dev)
    vol = tsdf.Volume.from_params(seq.volume)
    shape = choose_launch(vol, args, d, seq)
    maps = (torch.empty((H, W), device=dev), torch.empty((H, W, 3), device=dev), torch.empty((H, W, 3), device=dev))
    prm = {"iterations": args.icp_iterations}

    def step():
        vol.reset()
        est = [seq.poses[0].copy()]
        vol.fuse(d[0], seq.intr, est[0])
        for k in range(1, F):
            vol.raycast(seq.intr, est[-1], out=maps)
            pose, _ = vol.icp(d[k], seq.intr, maps[2], maps[1], est[-1], est[-1], prm)
            est.append(pose)
            vol.fuse(d[k], seq.intr, pose)
        return est

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        est = step()
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    clk = clocks.stop()
    vol.check()
    err = np.array([np.linalg.norm(est[k][:3, 3] - seq.poses[k][:3, 3]) for k in range(F)])
    ang = np.array([np.arccos(np.clip((np.trace(est[k][:3, :3] @ seq.poses[k][:3, :3].T) - 1) / 2, -1, 1))
                    for k in range(F)])
    # ICP alone, on the device and host, for one frame pair in the middle of the run
    k = F // 2
    vol.raycast(seq.intr, est[k - 1], out=maps)
    for _ in range(10):
        vol.icp(d[k], seq.intr, maps[2], maps[1], est[k - 1], est[k - 1], prm)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    reps = 100
    for _ in range(reps):
        vol.icp(d[k], seq.intr, maps[2], maps[1], est[k - 1], est[k - 1], prm)
    icp_ms = 1000.0 * (time.perf_counter() - t1) / reps
    line = {"metric": METRIC, "value": F * args.steps / sec, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 maps, f64 6x6 solve", "data": "synthetic",
            "config": {"workload": f"tracking: raycast -> point-to-plane ICP ({args.icp_iterations} iterations) -> "
                                   f"allocate -> integrate, 640x480, 2048^3 grid of 1.5 mm voxels, {F} frames",
                       "frames_per_step": F, "timing": "wall clock (ICP synchronises once per iteration)"},
            "launch": {"shape": shape},
            "tracking_error_mm": {"rms": float(1e3 * np.sqrt((err ** 2).mean())), "max": float(1e3 * err.max()),
                                  "final": float(1e3 * err[-1])},
            "tracking_error_deg": {"max": float(np.rad2deg(ang.max()))},
            "icp_ms_per_frame": icp_ms, "clocks": clk}
    vol.close()
    print(json.dumps(line), flush=True)


def run_mesh(args):
    """Marching-cubes extraction (tsdf_mesh) of the room volume after fusing
    the 300-frame sequence (640x480, 2048^3 grid of 1.5 mm voxels): one step =
    count + emit of the whole surface; triangles/s and ms per extraction, next
    to the raycast of one view of the same volume (the paper compares its two
    renderers)."""
    import numpy as np
    import torch

    from paper_1311_7194_b300 import build as pkg_build
    from paper_1311_7194_b300 import tsdf

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    pkg_build.build()
    seq = make_sequence(args.frames, dev, args.block_capacity)
    F, H, W = seq.depth.shape
    d = torch.from_numpy(seq.depth).to(dev)
    vol = tsdf.Volume.from_params(seq.volume)
    vol.set_launch_config(raycast_persistent=1)
    for k in range(F):
        vol.fuse(d[k], seq.intr, seq.poses[k])
    torch.cuda.synchronize()
    tri = None
    for _ in range(max(args.warmup, 0)):
        tri = vol.mesh()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        tri = vol.mesh()
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / args.steps
    clk = clocks.stop()
    maps = (torch.empty((H, W), device=dev), torch.empty((H, W, 3), device=dev), torch.empty((H, W, 3), device=dev))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        vol.raycast(seq.intr, seq.poses[-1], out=maps)
    e0.record()
    for _ in range(20):
        vol.raycast(seq.intr, seq.poses[-1], out=maps)
    e1.record()
    torch.cuda.synchronize()
    n = int(tri.shape[0])
    st = vol.stats()
    line = {"metric": "triangles/s", "value": n / sec, "unit": "triangles/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * sec, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"marching-cubes extraction of the room volume after {F} frames (2048^3 grid of "
                                   "1.5 mm voxels), count + emit, wall clock (synchronous call)",
                       "blocks": int(st["n_blocks"]), "triangles": n},
            "raycast_ms_one_view": e0.elapsed_time(e1) / 20, "clocks": clk}
    vol.close()
    print(json.dumps(line), flush=True)


def run_combined(args, emit=True):
    """The plain FP32 method against the form that stores T as FP16, fuses K = 8
    frames per graph launch and takes its measurement variances from the learned
    network, on the same GPU and sequence: the room (640x480, 2048^3 grid of
    1.5 mm voxels, 296 frames). For each form: frames/s, voxel updates/s and
    rays/s (the plain form raycasts every frame, the batched one every 8th), and
    the surface error of the fused model, i.e. the scene's analytic signed
    distance at the raycast vertices of four poses. The network is trained first
    (untimed) on room scenes with seeds 100-103 at the same size."""
    import numpy as np
    import torch

    from paper_1311_7194_b300 import build as pkg_build
    from paper_1311_7194_b300 import learned_variance as lv
    from paper_1311_7194_b300 import synth, tsdf

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    pkg_build.build()
    K = 8
    train_seqs = [synth.room_sequence(seed=sd, n_frames=40, device=dev) for sd in (100, 101, 102, 103)]
    data = lv.harvest(train_seqs, max_n=2_000_000, frame_stride=2)
    bits, hist = lv.train(data, steps=1500, batch=4096, lr=2e-3, seed=0)
    del train_seqs
    F = (args.frames // K) * K
    seq = make_sequence(F, dev, args.block_capacity)
    _, H, W = seq.depth.shape
    depth_dev = torch.from_numpy(seq.depth).to(dev)
    maps = (torch.empty((H, W), device=dev), torch.empty((H, W, 3), device=dev), torch.empty((H, W, 3), device=dev))
    eval_poses = [seq.poses[k] for k in (F // 5, 2 * F // 5, 3 * F // 5, F - 1)]
    forms = {"plain": dict(storage=tsdf.STORAGE_F32, K=1, mlp=None),
             "fp16_batched_learned": dict(storage=tsdf.STORAGE_F16, K=K, mlp=bits)}
    out = {}
    clocks = ClockSampler(0)
    for name, f in forms.items():
        vol = tsdf.Volume.from_params(seq.volume, storage=f["storage"])
        if not args.no_autotune:
            # launch shapes as the main workload picks them (results do not depend on them)
            vol.autotune([depth_dev[k] for k in range(20)], seq.intr, seq.poses[:20],
                         os.environ.get("TSDF_AUTOTUNE_CACHE"))
        if f["mlp"] is not None:
            vol.set_variance_mlp(f["mlp"])
        g = tsdf.Graph(vol, seq.intr, f["K"])
        k_ = f["K"]

        def step():
            vol.reset()
            for k in range(0, F, k_):
                g.launch([depth_dev[k + j] for j in range(k_)], seq.poses[k:k + k_], maps)

        for _ in range(max(args.warmup, 0)):
            step()
        torch.cuda.synchronize()
        vol.check()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(args.steps):
            step()
        t1.record()
        torch.cuda.synchronize()
        vol.check()
        sec = t0.elapsed_time(t1) / 1000.0
        st = vol.stats()
        err = lv.surface_error(vol, seq, eval_poses, seq.scene)
        out[name] = {"frames_per_s": F * args.steps / sec, "ms_per_step": 1000.0 * sec / args.steps,
                     "voxel_updates_per_s": st["voxel_updates_total"] * args.steps / sec,
                     "rays_per_s": (F // k_) * H * W * args.steps / sec, "raycast_every_n_frames": k_,
                     "surface_error_mm": {"mean_abs": 1e3 * err["mae"], "rms": 1e3 * err["rms"], "hits": err["hits"]},
                     "pool_bytes_per_voxel": (4 if f["storage"] == tsdf.STORAGE_F32 else 2) + 4}
        g.close()
        vol.close()
    clk = clocks.stop()
    comb, plain = out["fp16_batched_learned"], out["plain"]
    bound = 1.10
    line = {"metric": "frames/s", "value": comb["frames_per_s"], "unit": "frames/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": comb["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16 T / f32 P and arithmetic", "data": "synthetic",
            "config": {"workload": f"room 640x480, 2048^3 grid of 1.5 mm voxels, {F} frames: FP16 T + K={K} frames "
                                   "per graph launch + learned variance, against plain FP32 with one graph per frame",
                       "frames_per_step": F, "network_training": {"samples": data.n, "steps": 1500,
                                                                   "final_loss": hist[-1][1]}},
            "forms": out,
            "speedup_vs_plain": comb["frames_per_s"] / plain["frames_per_s"],
            "surface_error_bound": {"statement": f"mean surface error of the combined form within {bound:.2f}x "
                                                 "that of the plain FP32 form",
                                    "ratio": comb["surface_error_mm"]["mean_abs"] / plain["surface_error_mm"]["mean_abs"],
                                    "met": comb["surface_error_mm"]["mean_abs"]
                                    <= bound * plain["surface_error_mm"]["mean_abs"]},
            "clocks": clk}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_shift(args):
    """Volume shift with eviction (tsdf_shift / tsdf_import) on the room volume
    after fusing the 300-frame sequence (640x480, 2048^3 grid of 1.5 mm voxels):
    one step = shift the grid by 32 blocks along x (the blocks that leave it are
    copied to host memory), shift it back (block table rebuilt) and import the
    evicted blocks again, which restores the volume; blocks moved through host
    memory per second, wall clock (synchronous calls)."""
    import numpy as np
    import torch

    from paper_1311_7194_b300 import build as pkg_build
    from paper_1311_7194_b300 import tsdf

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    pkg_build.build()
    seq = make_sequence(args.frames, dev, args.block_capacity)
    F = seq.depth.shape[0]
    d = torch.from_numpy(seq.depth).to(dev)
    vol = tsdf.Volume.from_params(seq.volume)
    for k in range(F):
        vol.fuse(d[k], seq.intr, seq.poses[k])
    torch.cuda.synchronize()
    n_blocks = int(vol.stats()["n_blocks"])
    shift = (32, 0, 0)
    back = tuple(-x for x in shift)

    def step():
        t0 = time.perf_counter()
        ev = vol.shift(shift)
        t1 = time.perf_counter()
        vol.shift(back)
        t2 = time.perf_counter()
        vol.import_blocks(ev.coords, ev.T, ev.P)
        t3 = time.perf_counter()
        return len(ev.coords), (t1 - t0, t2 - t1, t3 - t2)

    for _ in range(max(args.warmup, 0)):
        step()
    clocks = ClockSampler(0)
    times = []
    moved = 0
    for _ in range(args.steps):
        m, t = step()
        moved = m
        times.append(t)
    clk = clocks.stop()
    times = np.asarray(times)
    sec = float(times.sum(1).mean())
    assert int(vol.stats()["n_blocks"]) == n_blocks
    line = {"metric": "blocks/s", "value": moved / sec, "unit": "evicted and re-imported blocks/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sec, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"volume shift of the room volume after {F} frames (2048^3 grid of 1.5 mm "
                                   "voxels) by 32 blocks along x and back, evicted blocks re-imported; wall clock",
                       "blocks": n_blocks, "evicted_per_step": moved,
                       "bytes_through_host_per_step": int(moved) * 512 * 8 * 2},
            "ms_shift_evict": 1000.0 * float(times[:, 0].mean()), "ms_shift_back": 1000.0 * float(times[:, 1].mean()),
            "ms_import": 1000.0 * float(times[:, 2].mean()), "clocks": clk}
    vol.close()
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "room" and dist_env()[2] > 1:
        raise SystemExit(f"--workload {args.workload} is a single-GPU measurement; run it without torchrun")
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload in ("capsules", "sphere"):
        run_capsules(args)
    elif args.workload == "tracking":
        run_tracking(args)
    elif args.workload == "mesh":
        run_mesh(args)
    elif args.workload == "shift":
        run_shift(args)
    elif args.workload == "combined":
        run_combined(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
