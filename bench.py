#!/usr/bin/env python
"""Benchmark of the render-and-score hot path: a coarse-to-fine multi-object parse.

One step = parse one synthetic tabletop scene (160x120 camera, table, box occluder, five
voxel objects of 2k-8k voxels at 5 mm): for each object in turn, the already-placed objects
are fixed at their inferred poses and the object's pose is enumerated coarse-to-fine
around a tracking prior: 3 stages x 9^3 translations x 200 rotations = 145,800 hypotheses
per stage, each rendered and scored under the windowed inlier-ball likelihood (r = 5 mm,
p_out = 0.01, 3x3 window), log-sum-exp normalised and resampled to 100 particles. That is
5 x 3 x 145,800 = 2,187,000 hypotheses per step, all on the device.

Prints one JSON line (rank 0). With --impl reference the CPU oracle is timed instead on a
bounded sample of the same workload (the reference arm).
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
import types

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2312_08715_gb300 import synth  # noqa: E402

METRIC = "pose hypotheses rendered+scored/sec on 1 GB300 (% HBM roofline); p99 frame latency"
UNIT = "hyp/s"
N_OBJECTS = 5
M_PARTICLES = 100
FIRST_SLOT = 2  # 0 = table, 1 = occluder

# FP32 operations per unit of counted work on the voxel-quad path of the score kernel, from
# the kernel source (an FMA counts 2):
#   corner: three lattice terms summed (6 ADD), 1/z, two projections (MUL + FMA each)
#   quad: signed area (edge function: 4 SUB, MUL, FMA), screen bbox (6 MIN, 6 MAX, 4 SUB),
#         affine 1/z plane (6 SUB, 2 FMA, 2 MUL, 2 DIV)
#   pixel test: four edge functions (4 x 7) + four sign products and tests
#   fragment: affine 1/z (2 FMA, 2 SUB), reciprocal, far test
#   composite pixel: min + test; scored pixel: ray row (3), lookup, delta, sum
#   window pair: ray column (ADD, SUB, MUL), offsets (2 FMA + SUB), |d|^2 (2 FMA + MUL), test
FLOPS_PER_UNIT = np.array([0.0, 13.0, 40.0, 36.0, 8.0, 2.0, 8.0, 14.0])
UNIT_NAMES = ["hypotheses", "corners", "primitives", "pixel_tests", "fragments", "composited_px",
              "scored_px", "window_pairs"]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b3d", choices=["b3d", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU work of the oracle baseline sample")
    ap.add_argument("--ref-seconds", type=float, default=30.0,
                    help="--impl reference: CPU work of the whole timed oracle run (warm-up included)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--mat-hyps", type=int, default=0,
                    help="materialised: the first N first-stage hypotheses only (0: all 145,800)")
    ap.add_argument("--no-materialised", action="store_true",
                    help="skip the render-then-score measurement appended to the default line")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving frame-latency leg appended to the default line")
    ap.add_argument("--trial", type=int, default=0)
    ap.add_argument("--workload", default="tabletop",
                    choices=["tabletop", "batched", "serving", "refine", "smc", "noise", "camera"],
                    help="batched: 64 independent scenes of uneven size in one captured CUDA graph of batched "
                         "launches per coarse-to-fine schedule, against looping the single-scene path; "
                         "serving: 32 concurrent tracking sessions through the server's continuous batching; "
                         "refine: gradient pose refinement (Adam) of 256 particles after coarse-to-fine enumeration; "
                         "smc: SMC over the object count, every particle its own coarse-to-fine proposal; "
                         "noise: one coarse-to-fine stage scored under a 4 x 4 grid of noise settings; "
                         "camera: camera-pose tracking of 120-frame videos at 25x25 to 200x200 (Table 1's setting)")
    ap.add_argument("--frames", type=int, default=40, help="serving: frames per session (warm-up included)")
    ap.add_argument("--sessions", type=int, default=32, help="serving: concurrent sessions")
    ap.add_argument("--linger-us", type=int, default=3000, help="serving: batch linger while a batch runs")
    ap.add_argument("--path", default="fused", choices=["fused", "materialised"],
                    help="materialised: render every first-stage hypothesis of the first object to HBM, "
                         "then score the stored images (the render-then-score form)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload(trial):
    return synth.tabletop_workload(trial, n_objects=N_OBJECTS)


def config_dict(wl, extra=None):
    c = dict(workload="coarse-to-fine tabletop parse: 160x120, 5 voxel objects (2k-8k voxels, 5 mm) + box "
                      "occluder + table, 3 stages x 9^3 translations x 200 rotations per object, 100 particles",
             hyps_per_step=N_OBJECTS * sum(s.n_per_axis ** 3 * s.n_rot for s in wl.stages),
             image=[wl.scene.camera.width, wl.scene.camera.height], likelihood="inlier ball r=5mm, p_out=0.01, 3x3",
             precision="fp32 kernels", l2="flushed between timed steps (256 MiB write)")
    if extra:
        c.update(extra)
    return c


# ------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------
_CLOCK_Q = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
            "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
            "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, uuid_hint=None):
        self.uuid_hint = uuid_hint
        self.proc = None
        self.path = os.path.join("/tmp", f"b3d_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={_CLOCK_Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            if self.uuid_hint and self.uuid_hint not in f[1]:
                continue
            rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------
# the GPU path
# ------------------------------------------------------------------------------------------
class Parse:
    """One multi-object coarse-to-fine parse through the C ABI (the timed step)."""

    def __init__(self, ctx, wl, torch):
        self.ctx, self.wl, self.torch = ctx, wl, torch
        sc = wl.scene
        self.ids = [ctx.load_mesh(m, closed=m.faces.shape[0] > 2) for m in sc.meshes]
        # known objects (table, occluder) at their true poses; objects at their tracking priors
        self.host_poses = np.array(sc.poses, np.float32)
        pri = wl.extra["priors"]
        for s in wl.extra["object_slots"]:
            self.host_poses[s] = pri[s]
        dev = ctx.device
        self.particles = torch.empty((N_OBJECTS, M_PARTICLES, 4, 4), dtype=torch.float32, device=dev)
        self.logw = torch.empty((N_OBJECTS, M_PARTICLES), dtype=torch.float32, device=dev)
        self.logq = torch.empty((N_OBJECTS, M_PARTICLES), dtype=torch.float32, device=dev)
        self.priors = pri

    def autotune(self, obs_dev):
        """Pick the score kernel's launch shape on the first object's first stage."""
        from paper_2312_08715_gb300 import b3d
        ctx, wl = self.ctx, self.wl
        b3d.b3d_set_scene(ctx.h, b3d.intrinsics(wl.scene.camera), self.ids[:FIRST_SLOT + 1],
                          self.host_poses[:FIRST_SLOT + 1], obs_dev, ctx.stream)
        return b3d.b3d_autotune(ctx.h, FIRST_SLOT, self.priors[FIRST_SLOT], wl.grid_frame,
                                b3d.stage_params(wl.stages[0]), b3d.lik_params(**wl.lik), ctx.stream)

    def run(self, obs_dev, seed=0):
        from paper_2312_08715_gb300 import b3d
        ctx, wl = self.ctx, self.wl
        for k in range(N_OBJECTS):
            slot = FIRST_SLOT + k
            b3d.b3d_set_scene(ctx.h, b3d.intrinsics(wl.scene.camera), self.ids[:slot + 1],
                              self.host_poses[:slot + 1], obs_dev, ctx.stream)
            for j in range(k):
                b3d.b3d_set_object_pose_dev(ctx.h, FIRST_SLOT + j, self.particles[j, 0], ctx.stream)
            ctx.enumerate_c2f(slot, self.priors[slot], wl.stages, wl.lik, M_PARTICLES, seed + 7919 * k,
                              wl.grid_frame, out=(self.particles[k], self.logw[k], self.logq[k]))


def gpu_observation(ctx, wl, torch):
    """Render the scene at its hidden poses on the GPU, then corrupt it with the seeded
    noise draws (host)."""
    sc = wl.scene
    ids = [ctx.load_mesh(m, closed=m.faces.shape[0] > 2) for m in sc.meshes]
    zeros = torch.zeros((sc.camera.height, sc.camera.width), dtype=torch.float32, device=ctx.device)
    ctx.set_scene(sc.camera, ids, sc.poses, zeros)
    depth, _ = ctx.render(FIRST_SLOT, sc.poses[FIRST_SLOT][None], want_tid=False)
    ctx.sync()
    return synth.corrupt_depth(depth[0].cpu().numpy(), sc.camera.far, wl.draws)


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2312_08715_gb300 import b3d
    b3d.load()

    wl = workload(args.trial + rank)  # each rank parses its own independent scene
    setup_ctx = b3d.Context(dev.index)
    obs_np = gpu_observation(setup_ctx, wl, torch)
    setup_ctx.close()

    ctx = b3d.Context(dev.index)
    parse = Parse(ctx, wl, torch)
    obs_dev = torch.as_tensor(obs_np, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    tuning = parse.autotune(obs_dev)  # untimed: launch shape of the score kernel

    # calibration (untimed): work counted by the kernels for one step
    b3d.b3d_set_instrumentation(ctx.h, b3d.B3D_INSTR_WORK)
    parse.run(obs_dev, seed=args.trial)
    ctx.sync()
    work = b3d.b3d_work_counters(ctx.h).astype(np.float64)
    b3d.b3d_set_instrumentation(ctx.h, 0)

    for w in range(args.warmup):
        parse.run(obs_dev, seed=args.trial + 100 + w)
    ctx.sync()

    # timed region: barrier + synchronize on both sides; per-step CUDA events; L2 flushed
    # before every step outside the events; per-kernel events recorded by the library.
    b3d.b3d_set_instrumentation(ctx.h, b3d.B3D_INSTR_TIMING)
    for k in range(b3d.B3D_K_COUNT):
        b3d.b3d_kernel_time(ctx.h, k)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    launches0 = ctx.launches()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(uuid) as clk:
        t_wall = time.perf_counter()
        for s in range(args.steps):
            flush.zero_()
            ev[s][0].record(stream)
            parse.run(obs_dev, seed=args.trial + 1000 + s)
            ev[s][1].record(stream)
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall
    ctx.sync()
    gpu_launches = ctx.launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    ktimes = {k: b3d.b3d_kernel_time(ctx.h, k) for k in range(b3d.B3D_K_COUNT)}
    b3d.b3d_set_instrumentation(ctx.h, 0)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())

    hyps_step = N_OBJECTS * sum(s.n_per_axis ** 3 * s.n_rot for s in wl.stages)
    value = hyps_step * args.steps * world / (total_ms / 1e3)
    px = wl.scene.camera.width * wl.scene.camera.height

    # roofline of the dominant kernel (the fused render+score kernel)
    score_ms, score_n = ktimes[b3d.B3D_K_SCORE]
    launches_per_step = N_OBJECTS * len(wl.stages)
    flop_per_launch = float(work @ FLOPS_PER_UNIT) / launches_per_step
    avg_launch_s = score_ms / max(score_n, 1) / 1e3
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    clocks = clk.summary()
    max_mhz = clocks.get("sm_max_mhz") or _measured_peaks().get("sm_max_mhz", 2070.0)
    peak_alu = n_sm * 128 * 2 * max_mhz * 1e6 / 1e12  # TFLOP/s: SMs x FP32 lanes x FMA x max SM clock
    achieved = flop_per_launch / avg_launch_s / 1e12
    traffic = _committed_traffic()
    hyps_per_launch = hyps_step / launches_per_step
    hbm_bytes_launch = (8.0 * px + 4.0) * hyps_per_launch
    peaks = _measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    e2e = None
    if rank == 0 and not args.no_e2e:
        e2e = run_e2e(args, ctx, parse, obs_np, flush, dev, torch, hyps_step)
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "ms_per_step_p50": float(np.percentile(step_ms, 50)), "ms_per_step_p99": float(np.percentile(step_ms, 99)),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_dict(wl, {"parallelism": f"replicas x{world} (independent scenes)",
                                   "score_kernel_tuning": tuning}),
        "px_hyps_per_s": value * px,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_alu, "unit": "TFLOP/s",
                     "frac": achieved / peak_alu, "traffic": traffic,
                     "kernel": "k_score<PoseGrid> (render + windowed likelihood)",
                     "avg_launch_ms": avg_launch_s * 1e3, "launches": score_n,
                     "flop_per_launch": flop_per_launch,
                     "peak_note": f"derived: {n_sm} SMs (device attribute) x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz "
                                  "(maximum SM clock, sampled)",
                     "work_per_step": {n: float(v) for n, v in zip(UNIT_NAMES, work)}},
        "hbm_equivalent": {"bytes_per_launch": hbm_bytes_launch,
                           "achieved_gbs": hbm_bytes_launch / avg_launch_s / 1e9, "peak_gbs": hbm_peak,
                           "frac": hbm_bytes_launch / avg_launch_s / 1e9 / hbm_peak,
                           "note": "materialised render-then-score traffic (8 B per pixel-hypothesis + 4 B per "
                                   "hypothesis) over the fused kernel's time, of measured HBM copy bandwidth"},
        "kernel_ms_per_step": {name: ktimes[k][0] / args.steps for k, name in enumerate(
            ["score", "render", "score_depth", "resample", "select", "grad", "scene"])},
        "gpu_launches": int(gpu_launches),
        "clocks": clocks,
        "wall_s_timed": t_wall,
    }
    if e2e:
        result["e2e"] = e2e
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args, wl, seconds=args.cpu_seconds)
    if world == 1 and not args.no_materialised:
        # the render-then-score form of the same first stage, measured after the timed region
        m = measure_materialised(wl, 3, 3, torch)
        result["materialised"] = {k: m[k] for k in ("ms_per_step", "hyp_per_s", "render", "score_depth", "hbm",
                                                    "agreement_with_fused")}
    if world == 1 and not args.no_serving:
        # the metric's frame latency: the serving workload (32 sessions at 320x240) for a few
        # frames per session, one frame in flight per camera, after the timed region
        result["serving"] = serving_leg()
    if rank == 0:
        print(json.dumps(result), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_e2e(args, ctx, parse, obs_np, flush, dev, torch, hyps_step):
    """End to end through the public API: every step copies its observation from pinned host
    memory to the device and reads the particles, weights and proposal densities back."""
    host_obs = torch.as_tensor(obs_np).pin_memory()
    dev_obs = torch.empty_like(host_obs, device=dev)
    outs = [parse.particles, parse.logw, parse.logq]
    host_out = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs]
    stream = torch.cuda.current_stream(dev)
    times = []
    for s in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        dev_obs.copy_(host_obs, non_blocking=True)
        parse.run(dev_obs, seed=args.trial + 5000 + s)
        for h, o in zip(host_out, outs):
            h.copy_(o, non_blocking=True)
        stream.synchronize()
        times.append(time.perf_counter() - t0)
    h2d = host_obs.numel() * 4
    d2h = sum(o.numel() * 4 for o in outs)
    return {"value": hyps_step * len(times) / sum(times), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * sum(times) / len(times),
            "p50_ms": 1e3 * float(np.percentile(times, 50)), "p99_ms": 1e3 * float(np.percentile(times, 99))}


def _measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _kernel_source_hash():
    h = hashlib.sha256()
    for f in ("k_score.cuh", "b3d_device.cuh", "b3d_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2312_08715_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _committed_traffic():
    """DRAM bytes per launch of the fused score kernel from the committed ncu summary, if
    it was taken from the current kernel source (else null)."""
    p = os.path.join(ROOT, "profiles", "fused_score_tabletop.json")
    try:
        d = json.load(open(p))
        if d.get("source_hash") == _kernel_source_hash():
            return d.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


# ------------------------------------------------------------------------------------------
# CPU oracle: baseline leg and reference arm
# ------------------------------------------------------------------------------------------
def _oracle_sample_inputs(wl):
    """First enumeration of the parse: object slot 2 in a scene of table + occluder + it,
    stage-1 grid around its tracking prior; observation rendered by the oracle."""
    from oracle import oracle as O
    sc = wl.scene
    full = O.render(sc)[0]
    obs = synth.corrupt_depth(full, sc.camera.far, wl.draws)
    sub = synth.Scene(sc.camera, sc.meshes[:FIRST_SLOT + 1], sc.poses[:FIRST_SLOT + 1].copy())
    st = wl.stages[0]
    rot = O.rotation_set(st.rot_kind, st.n_rot, st.rot_max)
    centre = wl.extra["priors"][FIRST_SLOT]
    poses = O.expand(centre, wl.grid_frame, st.n_per_axis, st.step, rot)
    return O, sub, obs, poses


def cpu_baseline(args, wl, seconds=12.0, label="oracle"):
    O, sub, obs, poses = _oracle_sample_inputs(wl)
    arrays = O.SceneArrays(sub)
    rng = np.random.default_rng(17)
    cores = O.max_threads()
    probe = poses[rng.choice(len(poses), 2 * cores, replace=False)]
    t0 = time.perf_counter()
    O.score(sub, FIRST_SLOT, probe, wl.lik, obs, flags=False, arrays=arrays)
    per = (time.perf_counter() - t0) / len(probe)
    n = int(min(len(poses), max(2 * cores, seconds / max(per, 1e-6))))
    sample = poses[rng.choice(len(poses), n, replace=False)]
    t0 = time.perf_counter()
    O.score(sub, FIRST_SLOT, sample, wl.lik, obs, flags=False, arrays=arrays)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} random hypotheses of the first stage of the first object (of 145,800; table + "
                      f"occluder + object, 160x120), FP64, OpenMP over hypotheses, {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = workload(args.trial)
    O, sub, obs, poses = _oracle_sample_inputs(wl)
    arrays = O.SceneArrays(sub)
    cores = O.max_threads()
    rng = np.random.default_rng(23)
    probe = poses[rng.choice(len(poses), 2 * cores, replace=False)]
    t0 = time.perf_counter()
    O.score(sub, FIRST_SLOT, probe, wl.lik, obs, flags=False, arrays=arrays)
    per = (time.perf_counter() - t0) / len(probe)
    # about --ref-seconds (30 s) of CPU work for the whole run, at least 1/20 of it per step
    step_s = max(args.ref_seconds / 20.0, args.ref_seconds / (args.warmup + args.steps))
    n_step = int(max(2 * cores, min(len(poses), step_s / max(per, 1e-6))))
    times = []
    for s in range(args.warmup + args.steps):
        sample = poses[rng.choice(len(poses), n_step, replace=False)]
        t0 = time.perf_counter()
        O.score(sub, FIRST_SLOT, sample, wl.lik, obs, flags=False, arrays=arrays)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = n_step * len(times) / sum(times)
    sample = (f"{n_step} random first-stage hypotheses per step (of 145,800), FP64 oracle, OpenMP over "
              f"{cores} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(wl, {"parallelism": "host cores"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def measure_materialised(wl, steps, warmup, torch, n_hyp=0):
    """The render-then-score form on the first stage of the first object: 145,800 depth
    images (160x120 float32, 11.2 GB) written to HBM by b3d_render_batch and read back by
    b3d_score_depth_batch. One step = both calls. Returns the measurement as a dict."""
    from paper_2312_08715_gb300 import b3d
    dev = torch.device("cuda", 0)
    setup_ctx = b3d.Context(0)
    obs_np = gpu_observation(setup_ctx, wl, torch)
    setup_ctx.close()
    ctx = b3d.Context(0)
    parse = Parse(ctx, wl, torch)
    obs_dev = torch.as_tensor(obs_np, device=dev)
    b3d.b3d_set_scene(ctx.h, b3d.intrinsics(wl.scene.camera), parse.ids[:FIRST_SLOT + 1],
                      parse.host_poses[:FIRST_SLOT + 1], obs_dev, ctx.stream)
    poses = ctx.expand(parse.priors[FIRST_SLOT], wl.grid_frame, wl.stages[0])
    if n_hyp > 0:
        poses = poses[:n_hyp].contiguous()
    n = poses.shape[0]
    H, W = wl.scene.camera.height, wl.scene.camera.width
    depth = torch.empty((n, H, W), dtype=torch.float32, device=dev)
    ll = torch.empty(n, dtype=torch.float32, device=dev)
    lik = b3d.lik_params(**wl.lik)
    stream = ctx.stream

    def step():
        b3d.b3d_render_batch(ctx.h, FIRST_SLOT, n, poses, depth, None, stream)
        b3d.b3d_score_depth_batch(ctx.h, FIRST_SLOT, n, depth, None, lik, ll, stream)

    for _ in range(warmup):
        step()
    ctx.sync()
    b3d.b3d_set_instrumentation(ctx.h, b3d.B3D_INSTR_TIMING)
    for k in range(b3d.B3D_K_COUNT):
        b3d.b3d_kernel_time(ctx.h, k)
    torch.cuda.synchronize(dev)
    a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler() as clk:
        a.record(stream)
        for _ in range(steps):
            step()
        b_.record(stream)
        torch.cuda.synchronize(dev)
    total_ms = a.elapsed_time(b_)
    r_ms, r_n = b3d.b3d_kernel_time(ctx.h, b3d.B3D_K_RENDER)
    s_ms, s_n = b3d.b3d_kernel_time(ctx.h, b3d.B3D_K_SCORE_DEPTH)
    b3d.b3d_set_instrumentation(ctx.h, 0)
    ctx.sync()
    # the same hypotheses through the fused kernel: the two forms agree to FP32 accuracy
    ll_fused = ctx.score(FIRST_SLOT, poses, wl.lik)
    ctx.sync()
    dll = (ll.double() - ll_fused.double()).abs()
    agree = {"max_abs": float(dll.max()), "median_abs": float(dll.median()),
             "max_rel": float((dll / ll_fused.double().abs().clamp_min(1.0)).max())}
    ctx.close()
    del depth
    px = H * W
    peak = _measured_peaks().get("hbm_gbs", 6800.0)
    wr = 4.0 * px * n / (r_ms / r_n / 1e3) / 1e9
    rd = (4.0 * px + 4.0) * n / (s_ms / s_n / 1e3) / 1e9
    ms = total_ms / steps
    return {"n": n, "ms_per_step": ms, "hyp_per_s": n / (ms / 1e3), "agreement_with_fused": agree,
            "render": {"ms": r_ms / r_n, "write_gbs": wr, "frac_of_hbm": wr / peak},
            "score_depth": {"ms": s_ms / s_n, "read_gbs": rd, "frac_of_hbm": rd / peak},
            "hbm": {"achieved_gbs": 8.0 * px * n / (ms / 1e3) / 1e9, "peak_gbs": peak,
                    "frac": 8.0 * px * n / (ms / 1e3) / 1e9 / peak,
                    "note": "8 B per pixel-hypothesis (4 B written + 4 B read) over the step, of measured HBM copy "
                            "bandwidth"},
            "clocks": clk.summary()}


def run_materialised(args):
    """The render-then-score form alone (see measure_materialised), as the bench line."""
    import torch
    wl = workload(args.trial)
    m = measure_materialised(wl, args.steps, args.warmup, torch, args.mat_hyps)
    print(json.dumps({
        "metric": METRIC, "value": m["hyp_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "path": "materialised",
        "config": config_dict(wl, {"workload": "render-then-score form: first stage of the first object "
                                               f"({m['n']} of its 145,800 hypotheses), depth images in HBM",
                                   "hyps_per_step": m["n"], "l2": "images exceed L2"}),
        "agreement_with_fused": m["agreement_with_fused"], "render": m["render"], "score_depth": m["score_depth"],
        "roofline": {"bound": "hbm", "achieved": m["hbm"]["achieved_gbs"], "peak": m["hbm"]["peak_gbs"],
                     "unit": "GB/s", "frac": m["hbm"]["frac"], "traffic": None, "note": m["hbm"]["note"]},
        "clocks": m["clocks"],
    }), flush=True)


def run_batched(args):
    """Batched form: 64 independent seeded scenes (1-8 objects, 500-20,000 voxels, 80x60 to
    320x240, 1,000-50,000 hypotheses per stage, log-uniform), two coarse-to-fine stages each.
    One step = the whole batch: replay of a captured CUDA graph of batched launches (3 per
    stage). Compared with looping b3d_enumerate_c2f over the scenes in the same launch shape."""
    import torch
    from paper_2312_08715_gb300 import b3d
    dev = torch.device("cuda", 0)
    wls = synth.batched_workloads(64)
    ctxs, items, outs = [], [], []
    M = 32
    for k, wl in enumerate(wls):
        ctx = b3d.Context(0)
        obs = gpu_observation(ctx, wl, torch)
        ids = list(range(len(wl.scene.meshes)))  # meshes were loaded in order by gpu_observation
        poses = np.array(wl.scene.poses, np.float32)
        poses[wl.slot] = wl.extra["priors"][wl.slot]
        ctx.set_scene(wl.scene.camera, ids, poses, obs)
        o = (torch.empty((M, 4, 4), device=dev), torch.empty(M, device=dev), torch.empty(M, device=dev))
        sch = b3d.schedule(wl.stages, M, 500 + k, wl.grid_frame)
        items.append(b3d.c2f_item(ctx.h, wl.slot, wl.extra["priors"][wl.slot], sch, *o))
        ctxs.append(ctx)
        outs.append(o)
    hyps_step = sum(sum(st.n_per_axis ** 3 * st.n_rot for st in wl.stages) for wl in wls)
    lik = b3d.lik_params(**wls[0].lik)
    owner = b3d.Context(0)
    big = max(range(len(wls)), key=lambda k: wls[k].scene.camera.width * wls[k].stages[0].n_rot)
    tuning = b3d.b3d_autotune(ctxs[big].h, wls[big].slot, wls[big].extra["priors"][wls[big].slot],
                              wls[big].grid_frame, b3d.stage_params(wls[big].stages[0]), lik, ctxs[big].stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def time_graph(g, n):
        ms = []
        for _ in range(n):
            flush.zero_()
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.replay()
            b_.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(a.elapsed_time(b_))
        return ms

    def capture(chunk, its=None):
        its = items if its is None else its
        t = dict(tuning, batch_chunk=chunk)
        b3d.b3d_set_tuning(owner.h, **t)
        b3d.b3d_enumerate_multi(owner.h, its, lik, owner.stream)  # sizes the scratch
        owner.sync()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                b3d.b3d_enumerate_multi(owner.h, its, lik, side)
        stream.wait_stream(side)
        return g

    # launch shape and batch chunk for the mix, picked by the library's batched autotuner
    # (timed on these items; the largest scene's single-stage pick need not suit the others)
    largest_pick = tuning
    b3d.b3d_set_tuning(owner.h, **tuning)
    tuning = b3d.b3d_autotune_multi(owner.h, items, lik, owner.stream)
    chunk = tuning["batch_chunk"]
    graph = capture(chunk)
    graph = capture(chunk)
    time_graph(graph, args.warmup)
    with ClockSampler() as clk:
        step_ms = time_graph(graph, args.steps)
    batched_ms = float(np.mean(step_ms))
    batched_out = [[t.clone() for t in o] for o in outs]
    # baseline: the single-scene path looped over the scenes, same launch shape
    for ctx in ctxs:
        b3d.b3d_set_tuning(ctx.h, **dict(tuning, batch_chunk=chunk))
    centres = [wl.extra["priors"][wl.slot] for wl in wls]

    def loop_once():
        for k, wl in enumerate(wls):
            ctxs[k].enumerate_c2f(wl.slot, centres[k], wl.stages, wl.lik, M, 500 + k, wl.grid_frame, out=outs[k])

    for _ in range(args.warmup):
        loop_once()
    torch.cuda.synchronize(dev)
    loop_ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        loop_once()
        b_.record(stream)
        torch.cuda.synchronize(dev)
        loop_ms.append(a.elapsed_time(b_))
    same = all(torch.equal(x, y) for bo, o in zip(batched_out, outs) for x, y in zip(bo, o))
    loop_mean = float(np.mean(loop_ms))
    small = _batched_small_scenes(args, wls, ctxs, owner, lik, capture, time_graph, chunk, flush, stream, torch, b3d,
                                  dev)
    print(json.dumps({
        "metric": METRIC, "value": hyps_step / (batched_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": batched_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "workload_kind": "batched",
        "config": {"workload": "batched form: 64 independent tabletop scenes (1-8 objects, 500-20,000 voxels, "
                               "80x60-320x240, 1,000-50,000 hypotheses per stage), 2 stages, 32 particles, one "
                               "CUDA graph of batched launches per step",
                   "hyps_per_step": hyps_step, "score_kernel_tuning": tuning, "batch_chunk": chunk,
                   "largest_scene_single_stage_pick": largest_pick,
                   "l2": "flushed between timed steps (256 MiB write)"},
        "loop_baseline": {"value": hyps_step / (loop_mean / 1e3), "ms_per_step": loop_mean,
                          "note": "b3d_enumerate_c2f looped over the 64 scenes (eager launches)"},
        "speedup_vs_loop": loop_mean / batched_ms, "outputs_equal_to_loop": bool(same),
        "small_scenes": small,
        "clocks": clk.summary(),
    }), flush=True)
    for c in ctxs + [owner]:
        c.close()

def _batched_small_scenes(args, wls, ctxs, owner, lik, capture, time_graph, chunk, flush, stream, torch, b3d, dev):
    """Where batching pays: the same 64 scenes with 1,000 hypotheses per stage (two stages of
    5^3 translations x 8 rotations, 8 particles), too few for one scene to fill the GPU: the
    batched graph against the single-scene calls looped over the scenes, same launch shape."""
    stages = [synth.StageSpec(5, 0.02, 1, 8, math.radians(8)), synth.StageSpec(5, 0.005, 1, 8, math.radians(2))]
    M = 8
    items, outs = [], []
    for k, wl in enumerate(wls):
        o = (torch.empty((M, 4, 4), device=dev), torch.empty(M, device=dev), torch.empty(M, device=dev))
        items.append(b3d.c2f_item(ctxs[k].h, wl.slot, wl.extra["priors"][wl.slot],
                                  b3d.schedule(stages, M, 900 + k, wl.grid_frame), *o))
        outs.append(o)
    g = capture(chunk, items)
    time_graph(g, max(1, args.warmup))
    batched_ms = float(np.mean(time_graph(g, args.steps)))
    batched_out = [[t.clone() for t in o] for o in outs]

    def loop_once():
        for k, wl in enumerate(wls):
            ctxs[k].enumerate_c2f(wl.slot, wl.extra["priors"][wl.slot], stages, wl.lik, M, 900 + k, wl.grid_frame,
                                  out=outs[k])

    for _ in range(max(1, args.warmup)):
        loop_once()
    torch.cuda.synchronize(dev)
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        loop_once()
        b_.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(a.elapsed_time(b_))
    loop_ms = float(np.mean(ms))
    hyps = len(wls) * sum(st.n_per_axis ** 3 * st.n_rot for st in stages)
    same = all(torch.equal(x, y) for bo, o in zip(batched_out, outs) for x, y in zip(bo, o))
    return {"workload": "the same 64 scenes, 2 stages of 1,000 hypotheses each, 8 particles", "hyps_per_step": hyps,
            "batched_ms": batched_ms, "batched_hyp_per_s": hyps / (batched_ms / 1e3), "loop_ms": loop_ms,
            "speedup_vs_loop": loop_ms / batched_ms, "outputs_equal_to_loop": bool(same)}


def _serving_streams(n_sessions, n_frames):
    """Session k tracks 1 + (k mod 6) objects (1-6, mean 3.5 over 32 sessions)."""
    return [synth.tracking_stream(k, n_objects=1 + k % 6, width=320, height=240, f=300.0, n_frames=n_frames)
            for k in range(n_sessions)]


def _serving_frames(streams, torch, dev):
    """Observed depth of every frame: the scene at its true poses rendered by the library
    (a camera stand-in: frames are inputs here, nothing is compared against them), then the
    seeded depth noise and outliers."""
    from paper_2312_08715_gb300 import b3d
    out = []
    for st in streams:
        ctx = b3d.Context(0)
        ids = [ctx.load_mesh(m, closed=m.faces.shape[0] > 2) for m in st.scene.meshes]
        blank = np.zeros((st.scene.camera.height, st.scene.camera.width), np.float32)
        frames = []
        for f in range(st.n_frames):
            ctx.set_scene(st.scene.camera, ids, st.truth[f], blank)
            depth, _ = ctx.render(0, st.truth[f][0:1], want_tid=False)
            frames.append(synth.corrupt_depth(depth[0].cpu().numpy(), st.scene.camera.far, st.draws(f)))
        ctx.close()
        out.append(frames)
    return out


def _serve(srv, sids, frames, first, last, fps, depth):
    """Drive the server like cameras: session s submits frames first..last-1, frame f at
    t0 + (f - first) / fps (fps 0: as soon as possible), with at most `depth` of its frames
    outstanding. Returns the frame results in completion order and the wall time from the
    first submission to the last result."""
    import heapq
    n = len(sids)
    F = last
    nxt = [first] * n
    out_k = [0] * n
    results = []
    period = 0.0 if fps <= 0 else 1.0 / fps
    t0 = time.perf_counter() + 0.002
    due = [(t0 + (k / n) * period, k) for k in range(n)]
    heapq.heapify(due)
    waiting = []  # sessions held back by the outstanding limit
    total = sum(F - first for _ in range(n))
    while len(results) < total:
        now = time.perf_counter()
        while due and due[0][0] <= now:
            _, k = heapq.heappop(due)
            if out_k[k] >= depth:
                waiting.append(k)
                continue
            srv.submit(sids[k], frames[k][nxt[k]], timeout_ms=60000)
            out_k[k] += 1
            nxt[k] += 1
            if nxt[k] < F:
                heapq.heappush(due, (max(now, t0 + (nxt[k] - first) * period + (k / n) * period), k))
        wait_ms = 50 if not due else max(0, min(50, int((due[0][0] - time.perf_counter()) * 1e3)))
        try:
            r = srv.next(wait_ms)
        except Exception as e:  # noqa: BLE001  (B3D_ETIMEOUT: nothing finished yet)
            if getattr(e, "status", None) != -5:
                raise
            continue
        results.append(r)
        k = sids.index(r["session"])
        out_k[k] -= 1
        if k in waiting:
            waiting.remove(k)
            heapq.heappush(due, (time.perf_counter(), k))
    return results, time.perf_counter() - t0


class ServingSetup:
    """The serving workload: 32 tracking sessions, each a 320x240 depth stream of 1-6 voxel
    objects moving on smooth random trajectories over a table (<= 1.7 cm and <= 4 degrees per
    frame). Per frame and tracked object: one enumeration of 5^3 translations (1 cm step, table
    axes) x 50 rotation perturbations (+-5 degrees) around the previous estimate, scored
    against the frame, with the other objects at their previous estimates; the best cell is
    the new estimate and 16 particles stay on the device. Sessions are admitted under a
    40 GB HBM budget; the server batches the frames of all sessions continuously."""

    def __init__(self, n_sessions, n_frames, linger_us):
        import torch
        from paper_2312_08715_gb300 import b3d
        self.b3d = b3d
        self.streams = _serving_streams(n_sessions, n_frames)
        self.frames = _serving_frames(self.streams, torch, torch.device("cuda", 0))
        self.lik = b3d.lik_params(kind=0, radius=0.005, p_outlier=0.01, half_window=1)
        self.stage = synth.tracking_stage(5, 0.01, 50, 5.0)
        self.sch = b3d.schedule([self.stage], 16, 0, np.eye(3))
        self.hyp_item = self.stage.n_per_axis ** 3 * self.stage.n_rot
        self.linger_us = linger_us
        # launch shape: autotuned on the session with the most objects
        big = max(range(len(self.streams)), key=lambda k: self.streams[k].n_track)
        st = self.streams[big]
        tctx = b3d.Context(0)
        ids = [tctx.load_mesh(m, closed=m.faces.shape[0] > 2) for m in st.scene.meshes]
        tctx.set_scene(st.scene.camera, ids, st.truth[0], self.frames[big][0])
        self.tuning = b3d.b3d_autotune(tctx.h, 0, st.truth[0][0], st.grid_frame, b3d.stage_params(self.stage),
                                       self.lik, tctx.stream)
        tctx.close()
        self.n_items = sum(s.n_track for s in self.streams)

    def serve(self, first, last, fps, max_batch_frames, depth=2):
        """Frames [0, first) as warm-up, then [first, last) timed, with at most `depth` frames in
        flight per camera (fps 0: each camera submits as soon as it may)."""
        b3d, streams, frames = self.b3d, self.streams, self.frames
        cfg = b3d.server_config(self.lik, self.sch, max_sessions=len(streams), max_batch_items=self.n_items,
                                max_inflight=2, queue_depth=4, tuning=dict(self.tuning),
                                max_batch_frames=max_batch_frames, batch_linger_us=self.linger_us)
        srv = b3d.Server(cfg, 0, 40 * 10 ** 9)
        sids = [srv.open_session(s.scene.camera, [(m.verts, m.faces) for m in s.scene.meshes], s.truth[0], s.n_track,
                                 s.seed, closed=[m.faces.shape[0] > 2 for m in s.scene.meshes],
                                 grid_frame=s.grid_frame) for s in streams]
        _serve(srv, sids, frames, 0, first, 0, depth)  # warm-up frames
        with ClockSampler() as clk:
            res, wall = _serve(srv, sids, frames, first, last, fps, depth)
        stats = srv.stats()
        srv.close()
        lat = np.array([r["latency_ms"] for r in res])
        hyps = sum(streams[sids.index(r["session"])].n_track for r in res) * self.hyp_item
        err = []
        for r in res:
            s = streams[sids.index(r["session"])]
            err.append(np.linalg.norm(r["poses"][:, :3, 3] - s.truth[r["frame_index"]][:s.n_track, :3, 3], axis=1))
        err = np.concatenate(err)
        poses = {(r["session"] - sids[0], r["frame_index"]): r["poses"] for r in res}
        return dict(hyp_per_s=hyps / wall, wall_s=wall, frames=len(res), p50_ms=float(np.percentile(lat, 50)),
                    p99_ms=float(np.percentile(lat, 99)), max_ms=float(lat.max()),
                    mean_batch_frames=float(np.mean([r["batch_frames"] for r in res])),
                    fps_per_session=len(res) / len(streams) / wall,
                    track_err_cm={"median": float(np.median(err) * 100), "p99": float(np.percentile(err, 99) * 100)},
                    hbm_reserved_gb=stats["hbm_reserved"] / 1e9, failed=stats["frames_failed"],
                    clocks=clk.summary()), poses

    def config(self, timed_frames):
        return {"workload": f"serving: {len(self.streams)} tracking sessions, 320x240 depth at 30 fps, 1-6 voxel "
                            "objects (2k-8k voxels, 5 mm) + table, per frame and object 5^3 x 50 = 6,250 "
                            "hypotheses around the previous estimate, 16 particles on the device, 40 GB budget",
                "sessions": len(self.streams), "tracked_objects": self.n_items, "hyps_per_object_frame": self.hyp_item,
                "frames_per_session": timed_frames, "score_kernel_tuning": self.tuning,
                "batch_linger_us": self.linger_us}


def serving_leg(frames_per_session=8, warmup=2, n_sessions=32):
    """The serving workload's frame latency for the default line (after its timed region): a
    bounded run with one frame in flight per camera."""
    setup = ServingSetup(n_sessions, warmup + frames_per_session, 3000)
    one, _ = setup.serve(warmup, warmup + frames_per_session, 0, 0, depth=1)
    return {"frame_p50_ms": one["p50_ms"], "frame_p99_ms": one["p99_ms"], "frame_max_ms": one["max_ms"],
            "hyp_per_s": one["hyp_per_s"], "frames": one["frames"], "fps_per_session": one["fps_per_session"],
            "mean_batch_frames": one["mean_batch_frames"], "track_err_cm": one["track_err_cm"],
            "frames_in_flight_per_session": 1, "clocks": one["clocks"],
            "config": setup.config(frames_per_session)}


def run_serving(args):
    """Serving form (see ServingSetup): throughput and per-frame latency with one frame in
    flight per camera, two in flight, cameras paced at 30 fps, and without cross-session
    batching."""
    W = max(1, min(args.warmup, args.frames - 1))
    setup = ServingSetup(args.sessions, args.frames, args.linger_us)
    # Each camera keeps one frame in flight (it submits frame f + 1 when frame f's result is
    # back): at saturation a frame's latency is the frames ahead of it over the throughput
    # (Little's law). Two in flight per camera gives the same throughput at twice the latency;
    # cameras paced at 30 fps (faster than the server) likewise queue two frames each.
    one, poses_one = setup.serve(W, args.frames, 0, 0, depth=1)
    sat, _ = setup.serve(W, args.frames, 0, 0)
    paced, _ = setup.serve(W, args.frames, 30.0, 0)
    solo, poses_solo = setup.serve(W, args.frames, 0, 1, depth=1)
    same = all(np.array_equal(poses_one[k], poses_solo[k]) for k in poses_one)
    cfg = setup.config(args.frames - W)
    cfg["step"] = "one frame of every session (value: aggregate throughput with one frame in flight per camera)"
    print(json.dumps({
        "metric": METRIC, "value": one["hyp_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.frames - W,
        "warmup": W, "ms_per_step": 1e3 * one["wall_s"] / (args.frames - W), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "workload_kind": "serving",
        "config": cfg,
        "latency_ms": {"p50": one["p50_ms"], "p99": one["p99_ms"], "frames_in_flight_per_session": 1},
        "one_frame_in_flight": one, "two_frames_in_flight": sat, "paced_30fps": paced,
        "no_cross_session_batching": solo,
        "speedup_vs_unbatched": one["hyp_per_s"] / solo["hyp_per_s"],
        "outputs_equal_to_unbatched": bool(same),
        "clocks": one["clocks"],
    }), flush=True)


def run_refine(args):
    """Differentiable form: the tabletop scene (160x120); the first object enumerated by the
    first two coarse-to-fine stages (2 x 145,800 hypotheses, 2 cm then 5 mm cells) to 256
    particles, then 50 Adam steps on each particle's se(3) pose under the smooth likelihood
    (Gaussian in 3D, sigma = 3 mm, p_out = 0.01, 5x5 window), forward and backward in one
    kernel per step: gradient refinement in place of the third, 1 mm stage (whose particles'
    error is reported beside). Also reported: the gradients with respect to sigma and p_out,
    and the forward-only throughput of the same likelihood."""
    import torch
    from paper_2312_08715_gb300 import b3d
    dev = torch.device("cuda", 0)
    wl = workload(args.trial)
    ctx = b3d.Context(0)
    obs = gpu_observation(ctx, wl, torch)
    ctx.set_scene(wl.scene.camera, list(range(len(wl.scene.meshes))), wl.scene.poses, obs)
    slot = FIRST_SLOT
    M, steps = 256, 50
    prior = wl.extra["priors"][slot]
    # refinement starts from the 256 particles of the full three-stage enumeration (2 cm, 5 mm,
    # 1 mm grids; each particle a drawn final cell moved uniformly within it)
    part3, _, _ = ctx.enumerate_c2f(slot, prior, wl.stages, wl.lik, M, 11, wl.grid_frame)
    T_start = part3.reshape(M, 4, 4).contiguous()
    part2, _, _ = ctx.enumerate_c2f(slot, prior, wl.stages[:2], wl.lik, M, 11, wl.grid_frame)
    T_two = part2.reshape(M, 4, 4).contiguous()
    smooth = dict(kind=1, radius=0.003, p_outlier=0.01, half_window=2)
    F = b3d.make_score_smooth()
    sigma = torch.tensor(smooth["radius"], device=dev, requires_grad=True)
    pout = torch.tensor(smooth["p_outlier"], device=dev, requires_grad=True)
    stream = torch.cuda.current_stream(dev)

    def refine(T):
        xi = torch.zeros((M, 6), device=dev, requires_grad=True)
        opt = torch.optim.Adam([xi], lr=3e-4)
        for _ in range(steps):
            opt.zero_grad(set_to_none=False)
            sigma.grad = None
            pout.grad = None
            ll = F.apply(xi, sigma, pout, ctx, slot, T, smooth["half_window"])
            (-ll.sum()).backward()
            opt.step()
            with torch.no_grad():
                T = ctx.se3_compose(xi, T)
                xi.zero_()
        return T

    for _ in range(max(1, args.warmup)):
        refine(T_start.clone())
    torch.cuda.synchronize(dev)
    ms = []
    with ClockSampler() as clk:
        for _ in range(args.steps):
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            T_end = refine(T_start.clone())
            b_.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(a.elapsed_time(b_))
    # the same refinement with one Adam step captured as a CUDA graph and replayed
    T_g = T_start.clone()
    xi_g = torch.zeros((M, 6), device=dev, requires_grad=True)
    opt_g = torch.optim.Adam([xi_g], lr=3e-4, capturable=True)

    def step_g():
        opt_g.zero_grad(set_to_none=False)
        ll = F.apply(xi_g, smooth["radius"], smooth["p_outlier"], ctx, slot, T_g, smooth["half_window"])
        (-ll.sum()).backward()
        opt_g.step()
        with torch.no_grad():
            ctx.se3_compose(xi_g, T_g, out=T_g)
            xi_g.zero_()

    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(3):
            step_g()
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step_g()
    gms = []
    for _ in range(args.steps):
        T_g.copy_(T_start)
        xi_g.data.zero_()
        for st_ in opt_g.state.values():
            for v in st_.values():
                if torch.is_tensor(v):
                    v.zero_()
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            graph.replay()
        b_.record(stream)
        torch.cuda.synchronize(dev)
        gms.append(a.elapsed_time(b_))
    ll_g = ctx.score(slot, T_g.clone(), smooth)
    # the same refinement through the library's entry point: every step in two kernels
    lib_ms = []
    for _ in range(3):
        ctx.refine(slot, T_start, smooth, steps, 3e-4)
    torch.cuda.synchronize(dev)
    for _ in range(args.steps):
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        T_lib, _ = ctx.refine(slot, T_start, smooth, steps, 3e-4)
        b_.record(stream)
        torch.cuda.synchronize(dev)
        lib_ms.append(a.elapsed_time(b_))
    ll_lib = ctx.score(slot, T_lib, smooth)
    # library kernel time of the forward + backward launches inside one refinement
    b3d.b3d_set_instrumentation(ctx.h, 1)
    refine(T_start.clone())
    torch.cuda.synchronize(dev)
    grad_ms, grad_n = b3d.b3d_kernel_time(ctx.h, 5)
    b3d.b3d_set_instrumentation(ctx.h, 0)
    # forward-only throughput of the same likelihood on the same 256 poses
    for _ in range(3):
        ctx.score(slot, T_start, smooth)
    torch.cuda.synchronize(dev)
    a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        ctx.score(slot, T_start, smooth)
    b_.record(stream)
    torch.cuda.synchronize(dev)
    fwd_ms = a.elapsed_time(b_) / steps
    ll0 = ctx.score(slot, T_start, smooth)
    ll1 = ctx.score(slot, T_end, smooth)
    hidden = wl.hidden[:3, 3]

    def t_err_mm(T):
        return np.linalg.norm(T[:, :3, 3].cpu().numpy() - hidden, axis=1) * 1e3

    def r_err_deg(T):
        R = T[:, :3, :3].cpu().numpy().astype(np.float64) @ wl.hidden[:3, :3].T.astype(np.float64)
        return np.degrees(np.arccos(np.clip((np.trace(R, axis1=1, axis2=2) - 1) / 2, -1, 1)))

    e0, e1 = t_err_mm(T_start), t_err_mm(T_end)
    # where does gradient refinement beat the 1 mm grid? library refinement over noise
    # scales and learning rates, from the same three-stage particles
    sweep = []
    for sig in (0.001, 0.002, 0.003):
        for lr in (3e-5, 1e-4, 3e-4, 1e-3):
            lk = dict(smooth, radius=sig)
            T_s, _ = ctx.refine(slot, T_start, lk, steps, lr)
            ls0, ls1 = ctx.score(slot, T_start, lk), ctx.score(slot, T_s, lk)
            sweep.append({"sigma_mm": sig * 1e3, "lr": lr, "median_t_err_mm": float(np.median(t_err_mm(T_s))),
                          "median_r_err_deg": float(np.median(r_err_deg(T_s))),
                          "loglik_gain_mean": float((ls1 - ls0).mean())})
    T_two_ref, _ = ctx.refine(slot, T_two, smooth, steps, 3e-4)
    # where the smooth likelihood's optimum lies: the same refinement from the true pose
    T_true = torch.as_tensor(np.repeat(wl.hidden[None].astype(np.float32), M, 0), device=dev)
    T_true_ref, _ = ctx.refine(slot, T_true, smooth, steps, 3e-4)
    xi = torch.zeros((M, 6), device=dev, requires_grad=True)
    sigma.grad = None
    pout.grad = None
    ll = F.apply(xi, sigma, pout, ctx, slot, T_end, smooth["half_window"])
    ll.sum().backward()
    mean_ms = float(np.mean(ms))
    print(json.dumps({
        "metric": METRIC, "value": M * steps / (mean_ms / 1e3), "unit": "hyp/s (forward+backward)", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "workload_kind": "refine",
        "config": {"workload": "differentiable refinement: tabletop 160x120, first object enumerated by three "
                               "coarse-to-fine stages (3 x 145,800 hypotheses, 2 cm, 5 mm, 1 mm) to 256 particles "
                               "(drawn cells jittered within the cell), then 50 Adam steps (lr 3e-4, se(3) re-based "
                               "each step) under the smooth likelihood sigma=3mm, p_out=0.01, 5x5",
                   "particles": M, "adam_steps": steps,
                   "step": "one whole refinement (50 forward+backward launches and the Adam updates)"},
        "grad_kernel_ms_per_launch": grad_ms / max(grad_n, 1),
        "graph_replay": {"ms_per_refinement": float(np.mean(gms)),
                         "hyp_per_s": M * steps / (float(np.mean(gms)) / 1e3),
                         "loglik_mean_after": float(ll_g.mean())},
        "library_refine": {"ms_per_refinement": float(np.mean(lib_ms)),
                           "hyp_per_s": M * steps / (float(np.mean(lib_ms)) / 1e3),
                           "loglik_mean_after": float(ll_lib.mean()),
                           "note": "b3d_refine_smooth: per step one forward+backward launch and one fused Adam + "
                                   "se(3) re-basing launch"},
        "forward_only": {"ms_per_launch": fwd_ms, "hyp_per_s": M / (fwd_ms / 1e3)},
        "loglik_mean": {"before": float(ll0.mean()), "after": float(ll1.mean()),
                        "improved_fraction": float((ll1 > ll0).float().mean())},
        "translation_error_mm": {"median_after_three_stages": float(np.median(e0)),
                                 "median_after_refinement": float(np.median(e1)),
                                 "from_two_stages": {"before": float(np.median(t_err_mm(T_two))),
                                                     "after_refinement": float(np.median(t_err_mm(T_two_ref)))},
                                 "from_the_true_pose_after_refinement": float(np.median(t_err_mm(T_true_ref)))},
        "rotation_error_deg": {"median_after_three_stages": float(np.median(r_err_deg(T_start))),
                               "median_after_refinement": float(np.median(r_err_deg(T_end)))},
        "refinement_sweep": sweep,
        "noise_gradients_at_end": {"dLL_dsigma": float(sigma.grad), "dLL_dpout": float(pout.grad)},
        "clocks": clk.summary(),
    }), flush=True)
    ctx.close()


def run_smc(args):
    """SMC over the number of objects (Sec. III-B, Eq. 2 and 3) on the tabletop scene: the
    five objects placed one per step by 16 particles, each proposing with its own
    coarse-to-fine search (3 stages x 145,800 hypotheses, path density as log q), re-scored
    at the proposal, weighted and resampled when the ESS drops below 8. One step = the whole
    parse: 5 x 16 x 437,400 = 35 million hypotheses."""
    import torch
    from paper_2312_08715_gb300 import b3d
    from paper_2312_08715_gb300.smc import SceneSMC
    dev = torch.device("cuda", 0)
    wl = workload(args.trial)
    sc = wl.scene
    ctx = b3d.Context(0)
    obs = gpu_observation(ctx, wl, torch)
    ctx.close()
    M = 16
    centres = [wl.extra["priors"][s] for s in wl.extra["object_slots"]]
    smc = SceneSMC(sc.camera, sc.meshes, sc.poses, [m.faces.shape[0] > 2 for m in sc.meshes], FIRST_SLOT, M)
    # launch shape: the autotuner's pick on the first object's first stage
    b3d.b3d_set_scene(smc.ctxs[0].h, b3d.intrinsics(sc.camera), smc.ids[0][:FIRST_SLOT + 1],
                      np.array(sc.poses[:FIRST_SLOT + 1], np.float32),
                      torch.as_tensor(obs, device=dev), smc.ctxs[0].stream)
    tuning = b3d.b3d_autotune(smc.ctxs[0].h, FIRST_SLOT, centres[0], wl.grid_frame, b3d.stage_params(wl.stages[0]),
                              b3d.lik_params(**wl.lik), smc.ctxs[0].stream)
    smc.set_tuning(**tuning)
    hyps = len(centres) * M * sum(s.n_per_axis ** 3 * s.n_rot for s in wl.stages)
    stream = torch.cuda.current_stream(dev)
    for w in range(max(1, args.warmup)):
        smc.run(obs, centres, wl.grid_frame, wl.lik, wl.stages, seed=100 + w)
    torch.cuda.synchronize(dev)
    ms, last = [], None
    with ClockSampler() as clk:
        for k in range(args.steps):
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            last = smc.run(obs, centres, wl.grid_frame, wl.lik, wl.stages, seed=k)
            b_.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(a.elapsed_time(b_))
    P, logw, log_ev, info = last
    w = torch.softmax(logw, 0).cpu().numpy()
    best = int(np.argmax(w))
    err = [float(np.linalg.norm(P[best, k, :3, 3].cpu().numpy() - sc.poses[s][:3, 3]) * 1e3)
           for k, s in enumerate(wl.extra["object_slots"])]
    mean_ms = float(np.mean(ms))
    smc.close()
    low = _smc_low_information(torch, b3d, SceneSMC, dev)
    print(json.dumps({
        "metric": METRIC, "value": hyps / (mean_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "workload_kind": "smc",
        "config": {"workload": "SMC over the object count: tabletop 160x120, 5 objects placed by 16 particles, each "
                               "its own coarse-to-fine proposal (3 stages x 145,800 hypotheses, path density), "
                               "resampling below ESS 8", "hyps_per_step": hyps, "particles": M,
                   "score_kernel_tuning": tuning},
        "ess_per_object": [round(i["ess"], 2) for i in info], "resampled": [i["resampled"] for i in info],
        "log_evidence": log_ev, "best_particle_translation_error_mm": err,
        "low_information": low,
        "clocks": clk.summary(),
    }), flush=True)


def _smc_low_information(torch, b3d, SceneSMC, dev):
    """The same sampler where the weights do not collapse (untimed beside the timed parse):
    the tabletop at 64x48 with table, occluder and two objects, the two placed by 16 particles
    under a 2 cm inlier ball with 10% outliers, three proposal stages (2 cm, 5 mm and 1 mm
    cells), resampling below ESS 12."""
    wl = synth.tabletop_workload(0, 5, 64, 48, 60.0)
    sc = synth.Scene(wl.scene.camera, wl.scene.meshes[:4], wl.scene.poses[:4].copy())
    ctx = b3d.Context(0)
    obs = gpu_observation(ctx, types.SimpleNamespace(scene=sc, draws=wl.draws), torch)
    ctx.close()
    stages = [synth.StageSpec(5, 0.02, 1, 4, math.radians(8)), synth.StageSpec(3, 0.005, 1, 2, math.radians(2)),
              synth.StageSpec(3, 0.001, 1, 2, math.radians(0.5))]
    centres = [wl.extra["priors"][2], wl.extra["priors"][3]]
    lik = dict(wl.lik, radius=0.02, p_outlier=0.1)
    M = 16
    smc = SceneSMC(sc.camera, sc.meshes, sc.poses, [m.faces.shape[0] > 2 for m in sc.meshes], FIRST_SLOT, M)
    smc.run(obs, centres, wl.grid_frame, lik, stages, seed=7, ess_frac=0.75)  # warm-up
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    P, logw, log_ev, info = smc.run(obs, centres, wl.grid_frame, lik, stages, seed=21, ess_frac=0.75)
    torch.cuda.synchronize(dev)
    ms = (time.perf_counter() - t0) * 1e3
    w = torch.softmax(logw, 0).cpu().numpy()
    smc.close()
    return {"workload": "tabletop 64x48 (table, occluder, 2 objects placed), inlier ball 2 cm, p_out 0.1, "
                        "3 stages (5^3 x 4 at 2 cm, 3^3 x 2 at 5 mm, 3^3 x 2 at 1 mm), 16 particles, "
                        "resampling below ESS 12",
            "ess_per_object": [round(i["ess"], 2) for i in info], "resampled": [i["resampled"] for i in info],
            "final_weight_max": float(w.max()), "final_ess": float(1.0 / np.sum(w ** 2)), "log_evidence": log_ev,
            "ms_wall": ms}


def run_noise(args):
    """Hierarchical noise (Alg. 1): the tabletop's first stage (145,800
    hypotheses of the first object) scored under a 4 x 4 grid of (inlier radius, outlier
    probability) settings in one fused pass, with the marginal over the grid; against the
    single-setting kernel on the same hypotheses."""
    import torch
    from paper_2312_08715_gb300 import b3d
    dev = torch.device("cuda", 0)
    wl = workload(args.trial)
    ctx = b3d.Context(0)
    obs = gpu_observation(ctx, wl, torch)
    sc = wl.scene
    ctx.set_scene(sc.camera, list(range(FIRST_SLOT + 1)), np.array(sc.poses[:FIRST_SLOT + 1], np.float32), obs)
    P = ctx.expand(wl.extra["priors"][FIRST_SLOT], wl.grid_frame, wl.stages[0])
    radii, pouts = [0.0025, 0.005, 0.01, 0.02], [0.001, 0.01, 0.1, 0.3]
    grid = b3d.noise_grid(0, radii, pouts, half_window=1)
    tuning = b3d.b3d_autotune(ctx.h, FIRST_SLOT, wl.extra["priors"][FIRST_SLOT], wl.grid_frame,
                              b3d.stage_params(wl.stages[0]), b3d.lik_params(**wl.lik), ctx.stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize(dev)
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b_.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(a.elapsed_time(b_))
        return float(np.mean(ms))

    with ClockSampler() as clk:
        grid_ms = timed(lambda: ctx.score_noise(FIRST_SLOT, P, grid))
        one_ms = timed(lambda: ctx.score(FIRST_SLOT, P, wl.lik))
    ll, marg = ctx.score_noise(FIRST_SLOT, P, grid)
    best = int(torch.argmax(marg))
    post = torch.softmax(ll[best].double(), 0).cpu().numpy().reshape(4, 4)
    n = P.shape[0]
    print(json.dumps({
        "metric": METRIC, "value": n / (grid_ms / 1e3), "unit": "hyp/s (16 noise settings each)", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": grid_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "workload_kind": "noise",
        "config": {"workload": "hierarchical noise: tabletop 160x120 first stage (145,800 hypotheses) under a 4 x 4 grid "
                               "of inlier radius {2.5, 5, 10, 20} mm x p_out {0.001, 0.01, 0.1, 0.3}, 3x3 window, "
                               "one fused pass + marginal", "score_kernel_tuning": tuning,
                   "l2": "flushed between timed steps (256 MiB write)"},
        "single_setting": {"ms_per_launch": one_ms, "hyp_per_s": n / (one_ms / 1e3)},
        "cost_of_16_settings_vs_1": grid_ms / one_ms,
        "noise_posterior_at_best_pose": {"radius_mm": [r * 1e3 for r in radii], "p_out": pouts,
                                         "p": post.round(4).tolist()},
        "clocks": clk.summary(),
    }), flush=True)
    ctx.close()


def run_camera(args):
    """Camera-pose tracking (Sec. IV, Table 1's setting): 3 synthetic objects x 4 image sizes
    (25x25 to 200x200), 120-frame videos of a camera panning around an object on a table,
    frame 0's pose given. Per frame a 6-stage search (2,048 rotations, then 27 translations,
    three times at finer scales: 6,225 camera poses), every
    hypothesis rendering the whole scene and scored on the full image. Reports frames per
    second (the whole per-frame loop, host included) and the pose error against the truth."""
    import torch
    from paper_2312_08715_gb300 import b3d
    from paper_2312_08715_gb300.camera import CameraTracker
    dev = torch.device("cuda", 0)
    lik = dict(kind=0, radius=0.005, p_outlier=0.01, half_window=1)
    stages = synth.camera_stages()
    rows = []
    n_frames = max(8, args.frames if args.frames != 40 else 120)
    with ClockSampler() as clk:
        for k in range(3):
            for size in (25, 50, 100, 200):
                v = synth.camera_video(k, size, n_frames=n_frames)
                closed = [True, False]
                # observations: the scene at the true camera poses, rendered by the library, plus noise
                r = b3d.Context(0)
                ids = [r.load_mesh(m, closed=c) for m, c in zip(v.scene.meshes, closed)]
                r.set_scene(v.scene.camera, ids, v.scene.poses, np.zeros((size, size), np.float32))
                clean, _ = r.render_camera(v.cam_from_world, want_tid=False)
                clean = clean.cpu().numpy()
                r.close()
                frames = [synth.corrupt_depth(clean[f], v.scene.camera.far, v.draws(f)) for f in range(v.n_frames)]
                tr = CameraTracker(v.scene.camera, v.scene.meshes, v.scene.poses, closed)
                est = v.cam_from_world[0]
                for f in range(1, min(4, v.n_frames)):  # warm-up on the first frames
                    tr.frame(frames[f], v.cam_from_world[f - 1], stages, lik, 32, f)
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                pos, ang = [], []
                for f in range(1, v.n_frames):
                    est, _ = tr.frame(frames[f], est, stages, lik, 32, f)
                    T, E = v.cam_from_world[f].astype(np.float64), est.astype(np.float64)
                    pos.append(np.linalg.norm(-T[:3, :3].T @ T[:3, 3] + E[:3, :3].T @ E[:3, 3]))
                    Rr = E[:3, :3] @ T[:3, :3].T
                    ang.append(math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(Rr) - 1) / 2)))))
                dt = time.perf_counter() - t0
                tr.close()
                nf = v.n_frames - 1
                pos_cm = np.array(pos) * 100
                rows.append({"object": k, "size": size, "fps": nf / dt,
                             "hyp_per_s": nf * sum(s.n_per_axis ** 3 * s.n_rot for s in stages) / dt,
                             "position_cm": float(np.mean(pos_cm)), "orientation_deg": float(np.mean(ang)),
                             "position_cm_median": float(np.median(pos_cm)),
                             "orientation_deg_median": float(np.median(ang)),
                             "frames_within_1cm": float(np.mean(pos_cm < 1.0))})
    fps200 = [r_["fps"] for r_ in rows if r_["size"] == 200]
    hps = float(np.mean([r_["hyp_per_s"] for r_ in rows]))
    print(json.dumps({
        "metric": METRIC, "value": hps, "unit": "hyp/s (camera hypotheses, full-image render + score)", "n_gpus": 1,
        "steps": n_frames - 1, "warmup": 3, "ms_per_step": 1e3 / float(np.mean([r_["fps"] for r_ in rows])),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "workload_kind": "camera",
        "config": {"workload": f"camera-pose tracking: 3 voxel objects on a table x 4 image sizes, {n_frames}-frame "
                               "panning videos, per frame 3 x (2,048 rotations + 27 translations) camera hypotheses (materialised render + "
                               "full-image score)", "step": "one video frame"},
        "per_video": rows, "fps_200x200_mean": float(np.mean(fps200)),
        "clocks": clk.summary(),
    }), flush=True)


def main():
    args = parse_args()
    if args.workload == "batched" and args.impl == "b3d":
        run_batched(args)
        return
    if args.workload == "serving" and args.impl == "b3d":
        run_serving(args)
        return
    if args.workload == "refine" and args.impl == "b3d":
        run_refine(args)
        return
    if args.workload == "smc" and args.impl == "b3d":
        run_smc(args)
        return
    if args.workload == "noise" and args.impl == "b3d":
        run_noise(args)
        return
    if args.workload == "camera" and args.impl == "b3d":
        run_camera(args)
        return
    if args.path == "materialised" and args.impl == "b3d":
        run_materialised(args)
        return
    if args.warmup < 3 and args.impl == "b3d":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
