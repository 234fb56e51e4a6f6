#!/usr/bin/env python
"""Benchmark of the batched environment step (Galactic, arXiv 2306.07552).

Metric: sim steps/sec = environments x steps / device time of the timed loop
(render + kinematics + collision, resets included at the workload's rate).
Default workload (uneven16384_nsdf, the full stack): 16384 envs over 64
procedural apartments with log-uniform 5k-150k triangles (2 cm distance
grid), 40 objects per env, 128x128 FP16 depth + RGB8, Gaussian actions,
Bernoulli(0.005) resets per env-step, and the per-scene neural SDF in the
static test (every scene's network trained before the timed loop by the
library's own kernels), timed beside the plain distance-grid form of the same
batch, with the share of contact decisions that differ between the two.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gx|reference]
                  [--workload NAME]

Under torchrun the global batch is N x the workload's environments (weak
scaling); rank g steps environments [g*E, (g+1)*E) of it, loads only the
scenes they use and draws its resets from the global environment indices;
no collective on the data path, per-step counters summed on the host; rank 0
prints one JSON line.  --impl reference times the FP64 CPU oracle on the host
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import contextlib
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2306_07552_b300 import inputs as I  # noqa: E402
from paper_2306_07552_b300 import shard  # noqa: E402

METRIC = "sim steps/sec (render+kinematics+collision) on 1 B300; fraction of roofline"
UNIT = "env-steps/s"
# Minimal per-unit work of the rasteriser in FP32/INT32 lane operations (one
# instruction of one lane; an FMA is one), for its ALU roofline.
# One front-facing triangle reaching the image:
#   half a vertex (closed meshes have ~T/2 vertices): P - eye 3, rotation to
#     camera space 9, reciprocal of z 1, projection 4, snap to 1/256 px 4
#     = 21, half of it                                                 10.5
#   facing: two edge vectors 6, their cross product 6, plane offset
#     n . (P0 - eye) 6, sign 1                                           19
#   screen edges dx, dy                                                   6
#   edge values at the first pixel centre (2 differences, 2 products
#     each)                                                              12
#   top-left bias                                                         6
#   bounding box: min/max of three per axis 8, to pixel centres 8, clamp
#     to the image 4                                                     20
#   depth plane: normal to camera space 9, 1/(h f) 2, coefficients 4    15
#   orientation from the doubled area, with the swap                      5
#   -> 93.5, rounded up
# One covered fragment: three edge values stepped 3, inside test 2, 1/z by
# one FMA 1, key (shift and or of the depth bits with colour and epoch) 3,
# framebuffer address 1, depth test 1 -> 11.
C_TRI = 94
C_FRAG = 11
LANES = 128          # FP32/INT32 lanes per SM


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 7:
                self.rows.append(p)

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [v for v in (num(r[0]) for r in self.rows) if v is not None]
        mx = [v for v in (num(r[1]) for r in self.rows) if v is not None]
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = [n for k, n in enumerate(self.NAMES)
                   if any(r[3 + k].lower() == "active" for r in self.rows)]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def golden(name):
    p = os.path.join(ROOT, "tests", "golden", name)
    return json.load(open(p)) if os.path.exists(p) else None


# Workloads whose views are drawn from another workload's scenes and camera
# statistics (the static test differs, the rendering work per view does not).
SAME_VIEWS = {"apartments4096_nsdf": "apartments4096", "uneven16384_nsdf": "uneven8192",
              "apartments4096_column": "apartments4096"}  # same scenes and cameras


def raster_work(workload):
    """Per-view triangles set up and fragments covered, measured by the
    oracle on a sample of the workload (written by oracle/raster_work.py)."""
    base = workload.split('-')[0]
    return golden(f"raster_work_{SAME_VIEWS.get(base, base)}.json")


def kernel_capture(workload, warps=None):
    """Per-launch figures of the rasteriser (DRAM bytes, warp instructions)
    scaled to the full workload from an ncu capture of a smaller case; None
    once the rasteriser source changed since the capture, or when the CTA
    shape timed (warps) is not the one captured."""
    p = os.path.join(ROOT, "profiles", f"raster_{workload}_traffic.json")
    if not os.path.exists(p):
        p = os.path.join(ROOT, "profiles",
                         f"raster_{SAME_VIEWS.get(workload, workload)}_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_sha1") != raster_source_sha1():
        return None
    if warps is not None and d.get("raster_warps") not in (None, warps):
        return None
    return d


def raster_source_sha1():
    """sha1 of the rasteriser's source (its kernel file, then its device code)."""
    csrc = os.path.join(ROOT, "paper_2306_07552_b300", "csrc")
    h = hashlib.sha1()
    for f in ("gx_raster.cu", "gx_raster_dev.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()


def kernel_traffic(workload, warps=None):
    d = kernel_capture(workload, warps)
    return d.get("bytes_per_launch_full") if d else None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2032.0)), "measured"
    return 6400.0, 2032.0, "fallback"


def loaded_clock_mhz():
    """Median SM clock of the B300s under a seconds-long dense load
    (written beside the measured peaks), or None."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(p):
        return None
    return json.load(open(p)).get("clocks_under_load", {}).get("sm_mhz_median")


def job_value(dist, n_envs, steps, ms_local):
    """Whole-job env-steps/s: all ranks' environments over the slowest rank's
    time (max over ranks)."""
    import torch
    world = dist.get_world_size() if dist else 1
    ms = ms_local
    if dist:
        t = torch.tensor([ms_local], dtype=torch.float64,
                         device="cuda" if dist.get_backend() == "nccl" else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * n_envs * steps / (ms / 1e3), ms


def reset_masks(n, period, first=0):
    """Staggered episodes of the global environments first .. first+n-1."""
    masks = np.zeros((period, n), np.uint8)
    for t in range(period):
        masks[t, (np.arange(first, first + n) + t) % period == 0] = 1
    return masks


def work_counters(ss, w, acts, mask_at, steps, plan, store):
    """Rasteriser work counters per view from a separate, untimed context
    running the counting variant of the kernel."""
    from paper_2306_07552_b300 import gx
    sim = gx.Sim(ss, I.fetch_like_robot(), w.n_envs, img=(w.img, w.img),
                 depth_fp16=w.depth_fp16, render_rgb=w.rgb, n_objects=w.n_objects,
                 obj_radius=w.obj_radius, seed=w.reset_seed, profile=3,
                 env_scene=plan.env_scene, env_offset=plan.first, static_store=store)
    sim.reset()
    for t in range(steps):
        sim.reset(mask_at(t))
        sim.step(acts[t])
    c = sim.raster_counters()
    sim.close()
    return {k: v / (steps * w.n_envs) for k, v in c.items()}


def object_mesh(w):
    """The oracle's instance mesh for the workload's objects."""
    return I.unit_cube() if w.objects == "boxes" else I.icosahedron()


def oracle_blank_state(w):
    """An empty oracle state in the workload's object model, ready for a reset."""
    import oracle as O
    st = O.Oracle.make_state((0, 0, 0), np.zeros(7))
    st.boxes = 1 if w.objects == "boxes" else 0
    return st


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_worker(args):
    """One host process: the oracle on its own disjoint set of environments
    for `seconds` of wall time; returns env-steps done."""
    wname, sample_envs, seconds = args
    w = I.WORKLOADS[wname]
    scenes = {}
    env_scene = I.env_scene_map(w.n_envs, w.n_scenes)
    targets = I.scene_tri_targets(w)
    import oracle as O
    robot = I.fetch_like_robot()
    states = []
    for e in sample_envs:
        s = int(env_scene[e])
        if s not in scenes:
            sc = (I.room_scene(w.scene_seed + s, targets[s], grid_h=w.grid_h)
                  if w.scene_kind == "room" else
                  I.apartment_scene(w.scene_seed + s, targets[s], grid_h=w.grid_h))
            scenes[s] = O.Oracle(robot, sc, object_mesh(w), I.object_colors(256))
        st = oracle_blank_state(w)
        scenes[s].reset(st, w.reset_seed, e, w.n_objects, *w.obj_radius)
        states.append((scenes[s], st))
    acts = I.make_actions(200, len(sample_envs), w.action_dist, seed=w.action_seed + 1)
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < seconds:
        k = done // len(sample_envs)
        for i, (orc, st) in enumerate(states):
            orc.step(st, acts[k % 200, i])
            orc.render(st, w.img, w.img)
            done += 1
    return done, time.perf_counter() - t0


def cpu_all_cores(w, seconds):
    """One oracle process per host core over disjoint environments (the
    environments are independent), started with spawn; aggregate rate."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    envs = np.linspace(0, w.n_envs - 1, 2 * cores).astype(int)
    jobs = [(w.name.split("-")[0], [int(envs[2 * c]), int(envs[2 * c + 1])], seconds)
            for c in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    rate = sum(d / t for d, t in res)
    return {"value": rate, "unit": UNIT, "cores": cores,
            "sample": f"{cores} processes x 2 envs each (disjoint), {seconds:.0f} s each, "
                      f"{sum(d for d, _ in res)} env-steps in all"}


def cpu_baseline(w, scenes, seconds):
    """The FP64 oracle on the host, single-threaded, on a bounded sample of
    the same workload: 8 envs spread over the scenes, reset, then stepped
    and rendered until `seconds` of CPU time are spent."""
    import oracle as O
    robot = I.fetch_like_robot()
    env_scene = I.env_scene_map(w.n_envs, w.n_scenes)
    sample_envs = [int(e) for e in np.linspace(0, w.n_envs - 1, 8)]
    orcs, states = {}, []
    for e in sample_envs:
        s = int(env_scene[e])
        if s not in orcs:
            orcs[s] = O.Oracle(robot, scenes[s], object_mesh(w), I.object_colors(256))
        st = oracle_blank_state(w)
        orcs[s].reset(st, w.reset_seed, e, w.n_objects, *w.obj_radius)
        states.append((orcs[s], st))
    acts = I.make_actions(200, len(sample_envs), w.action_dist, seed=w.action_seed + 1)
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < seconds and done < 200 * len(sample_envs):
        k = done // len(sample_envs)
        for i, (orc, st) in enumerate(states):
            orc.step(st, acts[k % 200, i])
            orc.render(st, w.img, w.img)
            done += 1
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} env-steps (physics + {w.img}x{w.img} render) over "
                      f"{len(sample_envs)} envs of {w.name}, {dt:.1f} s, one thread, FP64"
                      + ("; static test on the distance grid (the rule the neural form must "
                         "agree with)" if w.sdf == "neural" else ""),
            "cpu_model": cpu_model(), "nproc": os.cpu_count()}


# Neural SDF: algorithmic FLOPs per training sample (forward 64x128 +
# 3 x 128x128 + 128 MACs, backward-data 3 x 128x128, weight gradient 64x128 +
# 3 x 128x128; 2 FLOPs per MAC) and per query (forward only).
NSDF_TRAIN_FLOP = 2 * ((64 * 128 + 3 * 128 * 128 + 128) + 3 * 128 * 128 + (64 * 128 + 3 * 128 * 128))
NSDF_QUERY_FLOP = 2 * (64 * 128 + 3 * 128 * 128 + 128)
NSDF_BATCH = 65536
NSDF_BLOB_BYTES = 114688 + 2976


def train_scenes(ss, w, scenes_used):
    """Trains every used scene's network (untimed for the step metric);
    scenes_used: (index in the scene set, global scene index) pairs, the
    global index seeding the scene's sample stream.  Returns the training
    measurement.  The per-step time is the difference of a full and a short
    run on the first scene, so sample generation and workspace allocation
    cancel out."""
    B = I.fourier_matrix(w.nsdf_seed)
    P0 = I.nsdf_init(w.nsdf_seed)
    first, first_g = scenes_used[0]
    ss.nsdf_set_weights(first, B, P0)
    short = max(w.nsdf_steps // 4, 1)
    t0 = time.perf_counter()
    ss.nsdf_train(first, n_samples=w.nsdf_samples, batch=NSDF_BATCH, steps=short,
                  seed=w.nsdf_seed + first_g)
    t_short = time.perf_counter() - t0
    losses, total = [], 0.0
    for s, g in scenes_used:
        ss.nsdf_set_weights(s, B, P0)
        t0 = time.perf_counter()
        lo = ss.nsdf_train(s, n_samples=w.nsdf_samples, batch=NSDF_BATCH, steps=w.nsdf_steps,
                           seed=w.nsdf_seed + g)
        dt = time.perf_counter() - t0
        total += dt
        if s == first:
            t_full = dt
        losses.append(float(np.mean(lo[-20:])))
    step_ms = (t_full - t_short) / (w.nsdf_steps - short) * 1e3
    tflops = NSDF_BATCH * NSDF_TRAIN_FLOP / (step_ms / 1e3) / 1e12
    return {"scenes": len(scenes_used), "samples_per_scene": w.nsdf_samples,
            "batch": NSDF_BATCH, "adam_steps": w.nsdf_steps, "train_s_total": total,
            "step_ms": step_ms, "tflops": tflops,
            "final_loss_mean_m": float(np.mean(losses)),
            "flop_basis": f"{NSDF_TRAIN_FLOP} FLOP per sample (forward, backward-data, "
                          f"weight gradient)"}


def config_of(w):
    return {"workload": w.name, "envs": w.n_envs, "scenes": w.n_scenes,
            "triangles_per_scene": f"{w.tri_range[0]}-{w.tri_range[1]} {w.tri_dist}",
            "grid_h_m": w.grid_h, "objects": w.n_objects, "image": f"{w.img}x{w.img}",
            "depth": "f16" if w.depth_fp16 else "f32", "rgb8": w.rgb, "actions": w.action_dist,
            "resets": (f"{w.reset_every}-step episodes, staggered" if w.reset_every
                       else f"Bernoulli p={w.reset_prob} per env-step"),
            "l2": "no flush: each step writes more observation bytes than L2 holds",
            "object_model": w.objects,
            "static_test": {"neural": f"neural SDF, grid below {w.sdf_margin} m predicted "
                                      f"clearance",
                            "column": "column grid (radii 1.5/5/12 cm, 3 cm columns)"}.get(
                                w.sdf, "distance grid")}


def run_reference(args, w, rank, world):
    """Reference arm: the oracle as it stands, each step a bounded sample."""
    if rank != 0:
        return
    import oracle as O
    robot = I.fetch_like_robot()
    env_scene = I.env_scene_map(w.n_envs, w.n_scenes)
    sample = [int(e) for e in np.linspace(0, w.n_envs - 1, args.ref_envs)]
    used = sorted(set(int(env_scene[e]) for e in sample))
    scenes = dict(zip(used, I.make_scenes(w, only=used)))
    orcs, sts = {}, []
    for e in sample:
        s = int(env_scene[e])
        if s not in orcs:
            orcs[s] = O.Oracle(robot, scenes[s], object_mesh(w), I.object_colors(256))
        st = oracle_blank_state(w)
        orcs[s].reset(st, w.reset_seed, e, w.n_objects, *w.obj_radius)
        sts.append((orcs[s], st))
    acts = I.make_actions(args.warmup + args.steps, len(sample), w.action_dist,
                          seed=w.action_seed)

    def one(t):
        for i, (orc, st) in enumerate(sts):
            if w.reset_every and (t + sample[i]) % w.reset_every == 0:
                orc.reset(st, w.reset_seed, sample[i], w.n_objects, *w.obj_radius)
            orc.step(st, acts[t, i])
            orc.render(st, w.img, w.img)

    for t in range(args.warmup):
        one(t)
    t0 = time.perf_counter()
    for t in range(args.warmup, args.warmup + args.steps):
        one(t)
    dt = time.perf_counter() - t0
    value = len(sample) * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_of(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{len(sample)} envs of {w.name} per step, each step "
                                       f"physics + {w.img}x{w.img} render, FP64, one thread"
                                       + ("; static test on the distance grid (the rule the "
                                          "neural form must agree with)"
                                          if w.sdf == "neural" else "")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gx", choices=["gx", "reference"])
    ap.add_argument("--workload", default="uneven16384_nsdf", choices=list(I.WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-all-cores", type=float, default=8.0,
                    help="seconds of the all-cores oracle run (0: skip)")
    ap.add_argument("--no-counters", action="store_true")
    ap.add_argument("--ref-envs", type=int, default=4)
    ap.add_argument("--envs", type=int, default=0, help="smaller batch (profiling runs)")
    ap.add_argument("--scenes", type=int, default=0, help="fewer scenes (profiling runs)")
    ap.add_argument("--small-px", type=int, default=0, help="expansion bbox limit (0: auto)")
    ap.add_argument("--broadphase", action="store_true",
                    help="object broad-phase (four offset regular grids per environment)")
    ap.add_argument("--render-robot", action="store_true",
                    help="render the robot's collision spheres into every image")
    ap.add_argument("--heuristics", type=int, default=0,
                    help="the paper's heuristics: bit 0 sliding, bit 1 object placing")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default rasteriser setting instead of timing candidates")
    ap.add_argument("--occlusion", action="store_true",
                    help="cull clusters by occlusion (two phases per environment)")
    ap.add_argument("--fused", action="store_true",
                    help="one cooperative persistent launch per step (resets, physics, "
                         "rendering)")
    ap.add_argument("--no-graph", action="store_true",
                    help="headline from the event-timed loop instead of a graph-replayed one")
    ap.add_argument("--raster-warps", type=int, default=0, choices=[0, 6, 7, 8, 12],
                    help="warps per rasteriser CTA before autotuning (0: 7 where offered, else 8); with "
                         "--no-autotune the shape timed (profiling runs)")
    ap.add_argument("--static-store", type=int, default=-1, choices=[-1, 0, 1],
                    help="distance-grid nodes: 0 the dense grid, 1 the box store (recomputed "
                         "from the scene's boxes; the scene set then holds no dense grid); "
                         "-1: the box store for the neural form, else the dense grid")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()
    w = I.WORKLOADS[args.workload]
    if args.envs or args.scenes:
        w = dataclasses.replace(w, n_envs=args.envs or w.n_envs,
                                n_scenes=args.scenes or w.n_scenes,
                                name=f"{w.name}-{args.envs or w.n_envs}x{args.scenes or w.n_scenes}")
    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return

    import torch
    from paper_2306_07552_b300 import gx
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n = w.n_envs
    # this rank's shard of the global batch (world x n environments): its
    # environment range, the scenes those environments use, their map
    plan = shard.plan(world * n, w.n_scenes, world, rank)
    scenes = I.make_scenes(w, only=plan.scenes)
    neural = w.sdf == "neural"
    column = w.sdf == "column"
    store = args.static_store if args.static_store >= 0 else (1 if neural else 0)
    # with the box store the scene set holds no dense grid (nor, unless the
    # column form needs them, column grids): what the product keeps resident
    ss = (gx.SceneSet(scenes, dense_grid=False, column_grid=column) if store == 1
          else gx.SceneSet(scenes))
    nsdf = None
    if neural:
        nsdf = train_scenes(ss, w, list(enumerate(plan.scenes)))
    sim_kw = dict(img=(w.img, w.img), depth_fp16=w.depth_fp16, render_rgb=w.rgb,
                  n_objects=w.n_objects, obj_radius=w.obj_radius, seed=w.reset_seed,
                  small_tri_px=args.small_px, heuristics=args.heuristics,
                  render_robot=args.render_robot, broadphase=args.broadphase,
                  env_scene=plan.env_scene, env_offset=plan.first,
                  object_boxes=w.objects == "boxes", fused_step=args.fused,
                  occlusion_cull=args.occlusion, static_store=store,
                  raster_warps=args.raster_warps)
    sdf_mode = 1 if neural else (2 if column else 0)
    # per-kernel CUDA events on the launching stream (the roofline's kernel
    # time); the headline loop below replays the step as a CUDA graph on a
    # second context of the same batch
    sim = gx.Sim(ss, I.fetch_like_robot(), n, profile=1, sdf_mode=sdf_mode,
                 sdf_margin=w.sdf_margin, **sim_kw)
    total = args.warmup + args.steps
    # actions and reset draws of the global batch, this shard's columns
    sl = slice(plan.first, plan.first + n)
    acts = torch.from_numpy(np.ascontiguousarray(
        I.make_actions(total, world * n, w.action_dist, seed=w.action_seed)[:, sl])).cuda()
    if w.reset_every:
        masks_np = reset_masks(n, w.reset_every, plan.first)
        masks = torch.from_numpy(masks_np).cuda()
        mask_at = lambda t: masks[t % w.reset_every]  # noqa: E731
        host_mask = lambda t: masks_np[t % w.reset_every]  # noqa: E731
    else:
        rng = np.random.default_rng(w.reset_seed)
        mk_np = np.ascontiguousarray((rng.random((total + 2 * max(1, args.e2e_steps), world * n))
                                      < w.reset_prob).astype(np.uint8)[:, sl])
        mk = torch.from_numpy(mk_np).cuda()
        mask_at = lambda t: mk[t]  # noqa: E731
        host_mask = lambda t: mk_np[t]  # noqa: E731
    abuf = torch.empty((n, 11), dtype=torch.float32, device="cuda")
    mbuf = torch.empty((n,), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    launches = 0

    def one(ctx, t):
        # copy into fixed buffers so a graph replay sees the same pointers;
        # the step's resets and the step in one call (one graph, or with
        # --fused one kernel launch)
        abuf.copy_(acts[t])
        mbuf.copy_(mask_at(t))
        ctx.step_reset(mbuf, abuf, stream=stream)

    def warm(ctx):
        with torch.cuda.stream(stream):
            ctx.reset(stream=stream)
            for t in range(args.warmup):
                one(ctx, t)
            # device error bits of the warm-up (e.g. 0x2: a crowded reset kept
            # an object's last placement try), recorded and cleared
            err = ctx.device_error()
            tuned = None
            if not args.no_autotune:
                # rasteriser setting timed on this batch's own state (restored)
                abuf.copy_(acts[args.warmup - 1])
                tuned = ctx.autotune(abuf, steps=3, stream=stream)
        torch.cuda.synchronize()
        return err, tuned

    def timed(ctx, clk_on):
        """Steps warmup .. total-1 between two events on the launching
        stream, a barrier and a device synchronisation on both sides."""
        if dist:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) if clk_on else contextlib.nullcontext() as clk:
            torch.cuda.synchronize()
            e0.record(stream)
            with torch.cuda.stream(stream):
                for t in range(args.warmup, total):
                    one(ctx, t)
            e1.record(stream)
            torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return e0.elapsed_time(e1), clk

    warmup_err, tune = warm(sim)
    sim.phase_times()
    ms_events, clk_events = timed(sim, args.no_graph)
    phase_ms, phase_n = sim.phase_times()
    # the headline: the same steps of the same batch on a context that
    # replays each step as a captured CUDA graph (how a user runs it)
    gtune = None
    gsim = None
    if not args.no_graph:
        gsim = gx.Sim(ss, I.fetch_like_robot(), n, use_graph=True, sdf_mode=sdf_mode,
                      sdf_margin=w.sdf_margin, **sim_kw)
        _, gtune = warm(gsim)
        ms, clk = timed(gsim, True)
        dev_err = gsim.device_error()
        out_ctx = gsim
    else:
        ms, clk = ms_events, clk_events
        dev_err = sim.device_error()
        out_ctx = sim
    launches = args.steps * (1 if args.fused else (5 if neural else 3))
    value, ms = job_value(dist, n, args.steps, ms)
    value_events, _ = job_value(dist, n, args.steps, ms_events)
    # the last step's per-env results, summed over every rank's shard on the
    # host (a gloo group beside the NCCL one): no collective touches the step
    o = out_ctx.out
    last = {"env_steps": float(n), "contacts": float((o["contact_mask"] != 0).sum().item()),
            "grasps": float((o["event"] == 1).sum().item()),
            "releases": float(((o["event"] >= 3) & (o["event"] <= 5)).sum().item()),
            "reward_sum": float(o["reward"].double().sum().item())}
    shards = {"global_envs": world * n, "envs_per_rank": n, "rank0_envs": [plan.first, n],
              "rank0_scenes": list(plan.scenes),
              "last_step_summed": shard.sum_counters(
                  (dist, dist.new_group(backend="gloo")) if dist else None, last)}
    static_form = None

    def time_form(sset, **kw):
        """Another static form of the same batch, timed like the headline's
        event-timed loop: env-steps/s and physics ms per launch."""
        g = gx.Sim(sset, I.fetch_like_robot(), n, profile=1, **{**sim_kw, **kw})
        if tune:  # the event-timed loop's rasteriser setting: only the static form differs
            g.apply_tune(tune)
        with torch.cuda.stream(stream):
            g.reset(stream=stream)
            for t in range(args.warmup):
                abuf.copy_(acts[t])
                mbuf.copy_(mask_at(t))
                g.reset(mbuf, stream=stream)
                g.step(abuf, stream=stream)
        torch.cuda.synchronize()
        g.phase_times()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        with torch.cuda.stream(stream):
            for t in range(args.warmup, total):
                abuf.copy_(acts[t])
                mbuf.copy_(mask_at(t))
                g.reset(mbuf, stream=stream)
                g.step(abuf, stream=stream)
        g1.record(stream)
        torch.cuda.synchronize()
        v, _ = job_value(dist, n, args.steps, g0.elapsed_time(g1))
        g_ms, g_n = g.phase_times()
        g.close()
        return v, g_ms[0] / max(g_n[0], 1)

    if neural or column:
        # the plain distance-grid form of the same workload (dense grid)
        ss_dense = gx.SceneSet(scenes) if store == 1 else ss
        grid_value, grid_physics_ms = time_form(ss_dense, static_store=0, sdf_mode=0)
        if ss_dense is not ss:
            ss_dense.close()
        grid_bytes = [int(np.prod(sc.grid_dims)) * 4 for sc in scenes]
        if column:
            cb = [ss.column_info(s)[1] for s in range(len(scenes))]
            static_form = {"grid_form_value": grid_value,
                           "column_over_grid": value_events / grid_value,
                           "physics_ms": {"column": phase_ms[0] / max(phase_n[0], 1),
                                          "grid": grid_physics_ms},
                           "bytes_per_scene": {"grid_mean": float(np.mean(grid_bytes)),
                                               "column_mean": float(np.mean(cb))},
                           "note": "release, reset and the heuristics still read the grid"}
    if neural:
        # the method without the network but with the same small footprint:
        # every static test on the box store
        store_value, store_physics_ms = (time_form(ss, static_store=1, sdf_mode=0)
                                         if store == 1 else (None, None))
        sb = [ss.scene_bytes(s) for s in range(len(scenes))]
        hbm = torch.cuda.get_device_properties(0).total_memory
        render_mean = float(np.mean([b["render"] for b in sb]))
        store_mean = float(np.mean([b["box_store"] for b in sb]))
        static_neural = NSDF_BLOB_BYTES + (store_mean if store == 1 else np.mean(grid_bytes))
        # the neural form's decisions counted against the grid-only rule
        c = gx.Sim(ss, I.fetch_like_robot(), n, profile=4, sdf_mode=1, sdf_margin=w.sdf_margin,
                   **sim_kw)
        c.reset()
        for t in range(min(args.steps, 50)):
            c.reset(mask_at(t))
            c.step(acts[t])
        cnt = c.nsdf_counters()
        c.close()
        q_ms = phase_ms[3] / max(phase_n[3], 1)
        nsdf.update({
            "grid_form_value": grid_value, "neural_over_grid": value_events / grid_value,
            "static_store": ("box store: nodes recomputed from the scene's boxes; the scene set "
                             "holds no dense grid" if store == 1 else "dense grid"),
            "box_store_form_value": store_value,
            "neural_over_box_store": value_events / store_value if store_value else None,
            "physics_ms": {"neural": phase_ms[0] / max(phase_n[0], 1), "grid": grid_physics_ms,
                           "box_store": store_physics_ms},
            "query_ms_per_step": q_ms,
            "query_tflops": n * 32 * NSDF_QUERY_FLOP / (q_ms / 1e3) / 1e12 if q_ms else None,
            "query_flop_basis": f"{NSDF_QUERY_FLOP} FLOP per query, 32 query rows per env "
                                f"(31 used)",
            "decisions": cnt,
            "decisions_differing_from_grid": cnt["disagree"] / max(cnt["tests"], 1),
            "grid_consulted": cnt["grid_fallbacks"] / max(cnt["tests"], 1),
            "env_steps_differing": cnt["env_disagree"] / max(min(args.steps, 50) * n, 1),
            "bytes_per_scene": {"grid_mean": float(np.mean(grid_bytes)),
                                "network": NSDF_BLOB_BYTES, "box_store_mean": store_mean,
                                "render_mean": render_mean,
                                "static_neural_form": static_neural,
                                "static_grid_form": float(np.mean(grid_bytes))},
            "scenes_per_gpu": {
                "neural_form": int(hbm // (render_mean + static_neural)),
                "grid_form": int(hbm // (render_mean + np.mean(grid_bytes))),
                "note": f"{hbm / 2**30:.0f} GiB of HBM over one scene's render clusters and "
                        f"static structure (environment state and framebuffers aside)"},
            "note": ("below the margin the box store decides (the grid's node values "
                     "recomputed from the boxes), so no dense grid is resident"
                     if store == 1 else
                     "the dense grid stays resident: it decides every test below the margin")})

    # end to end through the C ABI with host buffers (pinned), copies inside
    # the timed region: actions in, the step's result (reward, success,
    # events) back; observations stay on the device for a GPU policy (the
    # paper's zero-copy hand-off).  Also timed: every output back to the host.
    # A user's context: the step replayed as a CUDA graph, no per-kernel
    # timing events, the rasteriser setting the autotuner picked for the
    # headline context (re-tuning here on three steps adds selection noise).
    sim.close()
    if gsim is not None:
        gsim.close()
    sim = gx.Sim(ss, I.fetch_like_robot(), n, profile=0, use_graph=True, sdf_mode=sdf_mode,
                 sdf_margin=w.sdf_margin, **sim_kw)
    with torch.cuda.stream(stream):
        sim.reset(stream=stream)
        for t in range(args.warmup):
            abuf.copy_(acts[t])
            mbuf.copy_(mask_at(t))
            sim.reset(mbuf, stream=stream)
            sim.step(abuf, stream=stream)
    if gtune or tune:
        sim.apply_tune(gtune or tune)
    torch.cuda.synchronize()
    full = sim.host_outputs(pinned=True)
    result = {k: (v if k in ("reward", "success", "event") else None) for k, v in full.items()}
    ne = max(1, args.e2e_steps)
    # each step's actions and reset mask wait in pinned host memory, where a
    # host-side policy would write them
    acts_h = torch.from_numpy(I.make_actions(2 * ne, n, w.action_dist,
                                             seed=w.action_seed + 99 + rank)).pin_memory()
    mask_h = torch.from_numpy(np.stack([host_mask(t) for t in range(2 * ne)])).pin_memory()

    def e2e_run(host, k0):
        sim.step_host(acts_h[k0], host, stream=stream)  # warm the path once
        t0 = time.perf_counter()
        for t in range(ne):
            # the workload's resets, their mask copied in from the host too
            with torch.cuda.stream(stream):
                mbuf.copy_(mask_h[k0 + t], non_blocking=True)
            sim.reset(mbuf, stream=stream)
            sim.step_host(acts_h[k0 + t], host, stream=stream)
        v, _ = job_value(dist, n, ne, (time.perf_counter() - t0) * 1e3)
        return v, int(sum(x.numel() * x.element_size() for x in host.values() if x is not None))

    e2e_value, d2h = e2e_run(result, 0)
    all_value, all_d2h = e2e_run(full, ne)
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * 11 * 4 + n,
           "d2h_bytes_per_step": d2h, "steps": ne,
           "note": "reset mask and actions in from pinned host memory, reset + "
                   "gx_step_host, reward/success/events back; observations stay on the "
                   "device (the paper's zero-copy hand-off to the policy)",
           "all_outputs": {"value": all_value, "d2h_bytes_per_step": all_d2h,
                           "note": "every output (images included) copied back each step"}}
    counters = None
    if rank == 0 and not args.no_counters:
        counters = work_counters(ss, w, acts, mask_at, min(args.warmup, 5), plan, store)
    sim.close()
    if rank != 0:
        ss.close()
        return

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, scenes, args.cpu_seconds)
        if args.cpu_all_cores > 0 and not (args.envs or args.scenes):
            cpu["all_cores"] = cpu_all_cores(w, args.cpu_all_cores)
    clocks = clk.summary()
    hbm_peak, sm_max_mhz, peak_src = measured_peaks()
    roof = None
    if phase_n[1]:
        launch_ms = phase_ms[1] / phase_n[1]
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        sm_mhz = clocks.get("sm_max_mhz") or sm_max_mhz
        peak = sms * LANES * sm_mhz * 1e6 / 1e12
        work = raster_work(w.name)
        achieved = no_cull = None
        if work:
            ops = n * (C_TRI * work["tris_per_view"] + C_FRAG * work["frags_per_view"])
            achieved = ops / (launch_ms / 1e3) / 1e12
            # upper bound of the work: every scene triangle set up in every view
            env_tris = np.array([scenes[s].n_tris for s in plan.env_scene])
            ops_all = C_TRI * env_tris.sum() + n * C_FRAG * work["frags_per_view"]
            no_cull = {"achieved": ops_all / (launch_ms / 1e3) / 1e12,
                       "frac": ops_all / (launch_ms / 1e3) / 1e12 / peak,
                       "note": "work if every scene triangle were set up in every view"}
        loaded = loaded_clock_mhz()
        at_loaded = None
        if loaded and achieved:
            p_l = sms * LANES * loaded * 1e6 / 1e12
            at_loaded = {"sm_mhz": loaded, "peak": p_l, "frac": achieved / p_l,
                         "note": "peak at the median SM clock of a seconds-long dense load "
                                 "(MEASURED_PEAKS.json); this run's own clocks are in 'clocks'"}
        # the rasteriser is instruction-bound: warp instructions issued per
        # second against 4 schedulers x 1 instruction per cycle per SM
        # the CTA shape timed: the tuned one, the one asked for, else the
        # library's default (7 warps, or 8 where the context needs them)
        shape = (tune["raster_warps"] if tune else args.raster_warps or
                 (8 if (args.fused or args.occlusion or w.objects == "boxes") else 7))
        cap = kernel_capture(w.name, shape)
        issue = None
        if cap and cap.get("warp_inst_per_launch_full"):
            rate = cap["warp_inst_per_launch_full"] / (launch_ms / 1e3) / 1e9
            pk = sms * 4 * sm_mhz * 1e6 / 1e9
            issue = {"warp_inst_per_launch": cap["warp_inst_per_launch_full"],
                     "achieved_ginst_s": rate, "peak_ginst_s": pk, "frac": rate / pk,
                     "note": "instructions from the ncu capture, scaled per environment; "
                             "the issue slots the kernel's own instruction stream fills"}
        obs = n * w.img * w.img * ((2 if w.depth_fp16 else 4) + (3 if w.rgb else 0))
        roof = {"bound": "alu", "kernel": "raster_kernel", "achieved": achieved, "peak": peak,
                "unit": "Tops/s (FP32/INT32 lane ops)",
                "frac": (achieved / peak) if achieved else None,
                "traffic": kernel_traffic(w.name, shape), "launch_ms": launch_ms,
                "raster_warps": shape,
                "peak_basis": f"{sms} SMs x {LANES} lanes x {sm_mhz:.0f} MHz ({peak_src} max "
                              f"clock)",
                "at_loaded_clock": at_loaded, "no_culling_bound": no_cull,
                "work_basis": f"{C_TRI} ops per front-facing triangle reaching the image + "
                              f"{C_FRAG} per covered fragment; counts per view from the oracle",
                "issue_view": issue,
                "hbm_view": {"bytes_per_launch": obs,
                             "achieved_gbs": obs / (launch_ms / 1e3) / 1e9,
                             "peak_gbs": hbm_peak, "peak_source": peak_src,
                             "frac": obs / (launch_ms / 1e3) / 1e9 / hbm_peak,
                             "note": "observation writes only"}}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (procedural apartments standing in for ReplicaCAD scenes, spheres for "
                "YCB objects, random actions for policy actions)",
        "config": {**config_of(w),
                   "step_launch": ("fused: one cooperative launch per step" if args.fused else
                                   "separate kernels: reset, physics, raster"),
                   "heuristics": {"sliding": bool(args.heuristics & 1),
                                                  "object_placing": bool(args.heuristics & 2)},
                   "robot_body_rendered": bool(args.render_robot),
                   "object_broadphase": bool(args.broadphase)},
        "timing": ("graph-replayed step (each step: reset launch + one graph replay), CUDA "
                   "events on the launching stream" if not args.no_graph else
                   "per-kernel CUDA events, no graph"),
        "event_timed": {"value": value_events, "ms_per_step": ms_events / args.steps,
                        "note": "the same steps on a context timing each kernel with CUDA "
                                "events (no graph); phases, the roofline and the static-form "
                                "ratios come from it"},
        "phases_ms_per_launch": {k: phase_ms[i] / max(phase_n[i], 1)
                                 for i, k in enumerate(["physics", "raster", "reset",
                                                        "nsdf_query"])},
        "nsdf": nsdf,
        "column_grid": static_form,
        "autotune": gtune or tune, "autotune_event_timed": tune,
        "shards": shards,
        "raster_counters_per_view": counters,
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches, "clocks": clocks, "device_error": dev_err,
        "device_error_warmup": warmup_err,
    }
    print(json.dumps(line), flush=True)
    ss.close()


if __name__ == "__main__":
    main()
