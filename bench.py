"""Benchmark: batched step + render of the uniform driving batch on B300 GPUs.

Workload (synthetic, seeded): 256 worlds x 32 agents (8192 cameras), 500 road segments
and 32 boxes per world, 128x128 uint8 class + FP32 depth per camera.  A step is one pass
of the whole hot path: the kinematic-bicycle/collision/off-road step of every world and
the render of every camera, replayed from a CUDA graph.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank simulates its own worlds (no
data-path collective; weak scaling); timings are max-reduced over ranks.
"""
import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import worldgen as wg  # noqa: E402

METRIC = "agent-steps/sec (step+render, 128x128) and Mpix/s vs plain FP32 path, same B300"
UNIT = "agent-steps/s"
WORKLOAD = wg.WORKLOADS["uniform"]
L2_BYTES = 126 * 2 ** 20
REASONS = {  # nvidia-smi clocks_event_reasons bit -> name
    0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
    0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
    0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting",
}


def workload_desc(wl, n_worlds):
    return ("uniform batch: %d worlds x %d agents (%d cameras), %d road segments and %d boxes "
            "per world, %dx%d uint8 class + fp32 depth" % (
                n_worlds, wl.agents[0], n_worlds * wl.agents[0], wl.segments[0], wl.boxes,
                wl.width, wl.height))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm,"
                 "clocks_event_reasons.active,power.draw", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 3:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                bits = int(r[2], 16) if r[2].startswith("0x") else int(r[2])
            except ValueError:
                continue
            for b, name in REASONS.items():
                if bits & b and name != "gpu_idle":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_worker(job):
    """One host core's share of the CPU baseline: from t_start, for `seconds`, step one of
    its worlds with the oracle and render every agent's camera, world after world."""
    worlds_list, wl, seconds, t_start, step = job
    import oracle
    cam = oracle.CamConfig(wl.width, wl.height, math.radians(wl.hfov_deg), wl.cam_height)
    sims = [oracle.Sim(one) for one in worlds_list]
    while time.time() < t_start:
        time.sleep(0.001)
    t_end = t_start + seconds
    done = 0
    w = 0
    while time.time() < t_end:
        sim = sims[w % len(sims)]
        sim.step(wg.actions(wl.seed, step + w // len(sims), sim.w.n_agents))
        for a in range(sim.w.n_agents):
            sim.render(cam, 0, a, 0.0)
            done += 1
            if time.time() >= t_end:
                break
        w += 1
    return done, time.time() - t_start


class OracleSampler:
    """The CPU oracle, as it stands, timed on a bounded sample of a workload on every host
    core: one spawned process per core (the bench process already holds a CUDA context),
    each stepping worlds of its own and rendering their cameras for a fixed wall time."""

    def __init__(self, worlds, wl, cores=None):
        import concurrent.futures
        import multiprocessing
        self.wl = wl
        self.cores = cores or host_cores()
        per = [[worlds.world(w % worlds.n_worlds) for w in range(j, j + 2 * self.cores, self.cores)]
               for j in range(self.cores)]
        self.per = per
        self.pool = concurrent.futures.ProcessPoolExecutor(
            self.cores, mp_context=multiprocessing.get_context("spawn"))
        # start every worker (imports, oracle library load) before the first timed sample
        list(self.pool.map(_oracle_worker, [([p[0]], wl, 0.0, 0.0, 0) for p in per]))

    def sample(self, seconds, step=0):
        """(agent-steps/s over all cores, wall seconds, agent cameras done)."""
        t_start = time.time() + 0.5
        res = list(self.pool.map(_oracle_worker,
                                 [(p, self.wl, seconds, t_start, step) for p in self.per]))
        done = sum(r[0] for r in res)
        wall = max(r[1] for r in res)
        return done / wall, wall, done

    def close(self):
        self.pool.shutdown()


def rank_workload(wl, rank):
    """This rank's own batch: the workload with a rank-specific seed.  Ranks share no data
    and exchange nothing on the data path (the worlds are independent)."""
    import dataclasses
    return dataclasses.replace(wl, seed=wl.seed + 7919 * rank)


def reduce_over_ranks(x, op, world, device):
    """x reduced over the ranks with torch.distributed op `op` ("max" or "sum")."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(total_agents, steps, max_ms):
    """Whole-job agent-steps/s: every rank's agents over the slowest rank's time."""
    return total_agents * steps / (max_ms / 1e3)


def accuracy_vs_oracle(sample):
    """Pixel-mismatch fraction and depth error of sampled GPU views against the CPU oracle's
    FP64 pipeline rendered from the same FP32 state: against the oracle in the path's own
    key precision (parity), and against its FP32-key image (the precision's error)."""
    import oracle
    worlds, wl, cfg = sample["worlds"], sample["wl"], sample["cfg"]
    o = oracle.Sim(worlds)
    o.set_state(sample["state"].astype(np.float64), sample["flags"])
    cam = oracle.CamConfig(int(cfg.width), int(cfg.height), float(np.float32(cfg.hfov)),
                           float(np.float32(cfg.cam_height)), float(np.float32(cfg.near_plane)),
                           float(np.float32(cfg.lane_line_z)))
    off = worlds.agent_offsets()
    f16 = bool(cfg.key_precision)
    onehot = int(cfg.output) == 1
    hot = None
    if onehot:
        hot = [int(oracle.f32_to_bf16_bits(np.float32((1 - np.float32(m)) / np.float32(sd)))[0])
               for m, sd in zip(cfg.norm_mean, cfg.norm_std)]
    mis_same = mis_f32 = total = 0
    rel, rel16 = [], []
    for k, v in enumerate(sample["views"]):
        agent, c = divmod(int(v), int(cfg.n_cams))
        w = int(np.searchsorted(off, agent, side="right") - 1)
        yaw = float(np.float32(cfg.cam_yaw[c]))
        g = sample["out"][k].numpy()
        if onehot:
            g16 = g.view(np.uint16)
            gcls = np.zeros(g16.shape[1:], np.uint8)
            for ch in range(4):
                gcls[g16[ch] == hot[ch]] = ch
        else:
            gcls = g
        gd = sample["depth"][k].numpy()
        gdepth = (gd.view(np.uint16).view(np.float16) if f16 else gd.view(np.float32)).astype(np.float64)
        ref32 = o.render(cam, w, agent - int(off[w]), yaw, False)
        ref = o.render(cam, w, agent - int(off[w]), yaw, True) if f16 else ref32

        def cls_of(img):
            return np.where(img.cls == 4, 3, img.cls) if onehot else img.cls
        mis_same += int((gcls != cls_of(ref)).sum())
        mis_f32 += int((gcls != cls_of(ref32)).sum())
        total += gcls.size
        both = (gcls > 0) & (gcls == cls_of(ref32))
        e = ref32.depth.astype(np.float64)
        if both.any():
            rel.append(np.abs(gdepth[both] - e[both]) / np.maximum(e[both], 1e-12))
        if f16:
            same = (gcls > 0) & (gcls == cls_of(ref))
            e16 = ref.depth.view(np.float16).astype(np.float64)
            if same.any():
                rel16.append(np.abs(gdepth[same] - e16[same]) / np.maximum(e16[same], 1e-12))
    r = np.concatenate(rel) if rel else np.zeros(1)
    out = {"views": int(len(sample["views"])), "pixels": int(total),
           "class_mismatch_frac_vs_oracle_same_precision": mis_same / max(total, 1),
           "class_mismatch_frac_vs_oracle_fp32_key": mis_f32 / max(total, 1),
           "depth_rel_err_vs_oracle_fp32_depth": {"max": float(r.max()), "p99": float(np.quantile(r, 0.99)),
                                                  "mean": float(r.mean())}}
    if f16:
        r16 = np.concatenate(rel16) if rel16 else np.zeros(1)
        out["depth_rel_err_vs_oracle_fp16_key"] = {"max": float(r16.max()), "mean": float(r16.mean())}
    return out


def algorithmic_bytes(sim, worlds, wl, with_depth=True):
    """The method's bytes per render launch (the hot path's own accounting): the
    images written, plus the world read once -- 32 B per road segment (stored as its
    parameters), about 40 B per agent (pose, size, speed, flags) and 28 B per static box."""
    n_w = worlds.n_worlds
    segs = int(wg.workload_counts(wl)[2][:n_w].sum())
    n_agents = int(worlds.n_agents)
    static = int(len(worlds.boxes)) - n_agents
    depth = sim.info.depth_bytes if with_depth else 0
    return sim.info.out_bytes + depth + 32 * segs + 40 * n_agents + 28 * static


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on all of this machine's host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOAD
    sampler = OracleSampler(wg.make_workload(wl, n_worlds=64), wl)
    # each step is a bounded sample; the whole run stays within a few minutes
    per_step = float(os.environ.get("GP_REF_STEP_SECONDS",
                                    str(min(5.0, max(0.5, 150.0 / (args.steps + args.warmup))))))
    for k in range(args.warmup):
        sampler.sample(min(per_step, 1.0), k)
    secs, agents = 0.0, 0
    for k in range(args.steps):
        r, el, n = sampler.sample(per_step, args.warmup + k)
        secs += el
        agents += n
    sampler.close()
    value = agents / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_desc(wl, wl.n_worlds)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": sampler.cores, "kind": "oracle",
                         "cpu": cpu_model(),
                         "sample": "each step: on every host core (one process each), worlds of "
                                   "the workload stepped and their cameras rendered one after "
                                   "another for %.2f s" % per_step},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def profiled_traffic(shape, kernel="render_kernel"):
    """DRAM bytes per launch of `kernel` from its committed ncu summary, if that capture was
    taken of the current render source at the same launch shape; else None."""
    import hashlib
    import re
    here = os.path.dirname(os.path.abspath(__file__))
    try:
        text = open(os.path.join(here, "profiles", kernel + "_uniform_128x128.md")).read()
        src = open(os.path.join(here, "paper_2606_19641_b300", "csrc", "gp_render.cu"), "rb").read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch: (\d+) \(render source sha256 ([0-9a-f]+), "
                  r"shape ([0-9a-z,]+)\)", text)
    if not m or m.group(3) != shape:
        return None
    if hashlib.sha256(src).hexdigest()[:len(m.group(2))] != m.group(2):
        return None
    return int(m.group(1))


PROFILE_CONFIGS = {
    # name: (workload, config overrides, depth plane written) -- as the bench times them
    "uniform": ("uniform", dict(), True),
    "uniform_precision": ("uniform", dict(key_precision=1, output=1), False),
    "ragged_precision_128x128": ("ragged", dict(key_precision=1, output=1), False),
    "ragged_precision_256x144": ("ragged_precision", dict(), False),
}


def run_profile(args):
    """One configuration's render, alone: --warmup then --steps direct render calls after
    one step; prints the mean render time (not a bench line)."""
    import torch
    from paper_2606_19641_b300 import Simulator, build, config_for
    build.build()
    name, _, nw = args.profile.partition(":")
    wl_name, kw, with_depth = PROFILE_CONFIGS[name]
    wl = wg.WORKLOADS[wl_name]
    worlds = wg.make_workload(wl, n_worlds=int(nw) if nw else None)
    shape = dict(autotune=1)
    if args.shape:
        rows, threads, cap = (int(v) for v in args.shape.split(","))
        shape = dict(band_rows=rows, threads=threads, tri_capacity=cap)
    sim = Simulator(worlds, config_for(wl, **shape, **kw))
    out, depth = sim.alloc_outputs(depth=with_depth)
    sim.step(torch.from_numpy(wg.actions(wl.seed, 0, worlds.n_agents)).cuda())
    for _ in range(args.warmup):
        sim.render(out, depth)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        sim.render(out, depth)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"profile": name, "worlds": worlds.n_worlds, "cameras": sim.n_views,
                      "render_ms": ms, "algorithmic_bytes": algorithmic_bytes(sim, worlds, wl, with_depth),
                      "shape": [sim.info.band_rows, sim.info.threads, sim.info.tri_capacity,
                                sim.info.producer_warps]}), flush=True)
    sim.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--backend", default="raster", choices=["raster", "trace"],
                    help="renderer of the timed step: the rasteriser (default) or the ray tracer")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the 3-camera resolution sweep 64..512 of both paths")
    ap.add_argument("--profile", default="",
                    help="profiling helper: NAME[:WORLDS] renders only that configuration "
                         "(uniform, uniform_precision, ragged_precision_128x128, "
                         "ragged_precision_256x144), --warmup then --steps direct render "
                         "calls, and prints their mean time; for ncu captures of a reduced batch")
    ap.add_argument("--shape", default="",
                    help="pin the render launch shape ROWS,THREADS,TRI_CAP instead of autotuning "
                         "(for profiler captures that must skip a known number of launches)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)

    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2606_19641_b300 import Simulator, build, config_for
    build.build()

    wl = WORKLOAD
    # each rank simulates its own batch of worlds (different seed): no data-path collective
    wl_rank = rank_workload(wl, rank)
    worlds = wg.make_workload(wl_rank)
    if args.shape:
        rows, threads, cap = (int(v) for v in args.shape.split(","))
        shape = dict(band_rows=rows, threads=threads, tri_capacity=cap)
    else:
        shape = dict(autotune=1)
    sim = Simulator(worlds, config_for(wl_rank, **shape), device=local)
    out, depth = sim.alloc_outputs()
    n_agents = sim.n_agents
    px = wl.width * wl.height
    stream = torch.cuda.current_stream()

    acts = [torch.from_numpy(wg.actions(wl_rank.seed, k, n_agents)).cuda()
            for k in range(args.warmup + args.steps)]
    act = torch.empty_like(acts[0])
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def maxred(x):
        return reduce_over_ranks(x, "max", world, "cuda")

    trace = args.backend == "trace"
    step_render = sim.step_trace if trace else sim.step_render
    render = sim.trace if trace else sim.render

    # warm-up (graph capture happens on the first replay)
    for k in range(args.warmup):
        act.copy_(acts[k])
        step_render(act, out, depth)
    barrier()

    # --- timed: graph replays of step+render, L2 evicted between steps (not timed) ---
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        for k in range(args.steps):
            act.copy_(acts[args.warmup + k])
            flush.fill_(float(k))
            ev[k][0].record(stream)
            step_render(act, out, depth)
            ev[k][1].record(stream)
        barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = maxred(sum(step_ms))
    ms_per_step = total_ms / args.steps
    total_agents = reduce_over_ranks(n_agents, "sum", world, "cuda")
    value = job_rate(total_agents, args.steps, total_ms)

    # --- render-kernel time inside a timed loop of direct calls (roofline) ---
    evr = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        act.copy_(acts[args.warmup + k])
        flush.fill_(float(k))
        evr[k][0].record(stream)
        sim.step(act)
        evr[k][1].record(stream)
        render(out, depth)
        evr[k][2].record(stream)
    barrier()
    render_ms = statistics.mean(b.elapsed_time(c) for a, b, c in evr)
    stepk_ms = statistics.mean(a.elapsed_time(b) for a, b, c in evr)
    out_bytes = sim.info.out_bytes + sim.info.depth_bytes
    algo_bytes = algorithmic_bytes(sim, worlds, wl_rank)
    peak, peak_kind = peaks()
    achieved = algo_bytes / (render_ms / 1e3) / 1e9
    shape_s = "%d,%d,%d" % (sim.info.band_rows, sim.info.threads, sim.info.tri_capacity)
    kernel = "trace_kernel" if trace else "render_kernel"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": profiled_traffic("trace" if trace else shape_s, kernel),
                "kernel": kernel,
                "peak_source": peak_kind, "algorithmic_bytes_per_launch": algo_bytes,
                "avg_launch_ms": render_ms, "frac_of_nominal_8tbs": achieved / 8000.0}

    # --- end to end through the C ABI with host buffers ---
    # every step's actions wait in pinned host memory (as a policy on the host would hand
    # them over); the timed loop copies them in and reads the state back each step
    e2e_steps = min(args.steps, 50)
    h_acts = torch.from_numpy(np.stack([wg.actions(wl_rank.seed, k, n_agents)
                                        for k in range(e2e_steps)])).pin_memory()
    h_act = h_acts[0]
    h_state = torch.empty((n_agents, 4), dtype=torch.float32).pin_memory()
    h_flags = torch.empty((n_agents,), dtype=torch.uint8).pin_memory()
    d_state = torch.empty((n_agents, 4), dtype=torch.float32, device="cuda")
    d_flags = torch.empty((n_agents,), dtype=torch.uint8, device="cuda")
    if not trace:  # untimed: the host call's graph (keyed on its staging buffer) is captured here
        sim.step_render_host(h_acts[0], out, depth, h_state, h_flags, stream=stream)
        stream.synchronize()
    barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        if trace:  # five calls: copy in, step + trace, state export, two copies out
            act.copy_(h_acts[k], non_blocking=True)
            step_render(act, out, depth)
            sim.get_state_device(d_state, d_flags)
            h_state.copy_(d_state, non_blocking=True)
            h_flags.copy_(d_flags, non_blocking=True)
        else:  # one call: gp_step_render_host
            sim.step_render_host(h_acts[k], out, depth, h_state, h_flags, stream=stream)
        stream.synchronize()
    e2e_s = maxred(time.perf_counter() - t0)
    e2e = {"value": job_rate(total_agents, e2e_steps, 1e3 * e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": h_act.numel() * 4,
           "d2h_bytes_per_step": h_state.numel() * 4 + h_flags.numel(),
           "note": "actions host->device and agent state/flags device->host every step "
                   "(one gp_step_render_host call per step for the raster), the host waiting "
                   "for each step's state; images stay on the GPU as a batched tensor; no L2 "
                   "flush between steps (each step writes 671 MB of images, 5x the L2)"}

    extras = {}

    # GPU images of sampled views for the accuracy check of the CPU leg (the oracle renders
    # the same views from the same FP32 state after every GPU timing is done)
    accuracy_samples = {}

    def keep_sample(key, sim2, worlds2, wl2, n_views=64):
        o2, d2 = sim2.alloc_outputs(depth=True)
        sim2.render(o2, d2)
        torch.cuda.synchronize()
        views = np.unique(np.linspace(0, sim2.n_views - 1, n_views).round().astype(np.int64))
        st, fl = sim2.get_state()
        idx = torch.from_numpy(views).cuda()

        def bits(t):  # raw bits (numpy has no bfloat16)
            return t.view(torch.int16) if t.element_size() == 2 else (
                t.view(torch.int32) if t.element_size() == 4 else t)
        accuracy_samples[key] = dict(
            worlds=worlds2, wl=wl2, cfg=sim2.config, views=views, state=st, flags=fl,
            out=bits(o2[idx]).cpu(), depth=bits(d2[idx]).cpu())
        del o2, d2

    def graph_rate(sim2, worlds2, wl2, steps, depth=False):
        """agent-steps/s and render roofline of graph replays for another configuration."""
        o2, d2 = sim2.alloc_outputs(depth=depth)
        a2 = [torch.from_numpy(wg.actions(wl2.seed, k, sim2.n_agents)).cuda() for k in range(steps + 3)]
        for k in range(3):
            sim2.step_render(a2[k], o2, d2)
        barrier()
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for k in range(steps):
            flush.fill_(float(k))
            ev2[k][0].record(stream)
            sim2.step_render(a2[3 + k], o2, d2)
            ev2[k][1].record(stream)
        barrier()
        ms = maxred(sum(a.elapsed_time(b) for a, b in ev2)) / steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        for k in range(steps):
            sim2.render(o2, d2)
        e1.record(stream)
        barrier()
        rms = e0.elapsed_time(e1) / steps
        rb = algorithmic_bytes(sim2, worlds2, wl2, with_depth=depth)
        agents2 = reduce_over_ranks(sim2.n_agents, "sum", world, "cuda")
        del o2, d2
        return {"agent_steps_per_s": job_rate(agents2, 1, ms), "ms_per_step": ms,
                "render_kernel_ms": rms, "render_gbs": rb / (rms / 1e3) / 1e9,
                "render_frac_of_measured_hbm": rb / (rms / 1e3) / 1e9 / peaks()[0],
                "cameras": sim2.n_views, "band_rows": sim2.info.band_rows,
                "threads": sim2.info.threads, "tri_capacity": sim2.info.tri_capacity,
                "planes_written": ("the output tensor and the depth plane" if depth
                                   else "the output tensor only (no depth plane)")}

    if not args.no_extras:
        keep_sample("uniform_fp32_u8_class", sim, worlds, wl_rank)
        # plain per-world path: one step launch and one render launch per world, no graph
        pw_steps = 5
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(pw_steps):
            for w in range(worlds.n_worlds):
                sim.step_world(w, act)
            for w in range(worlds.n_worlds):
                sim.render_world(w, out, depth)
        e1.record(stream)
        barrier()
        pw_ms = maxred(e0.elapsed_time(e1)) / pw_steps
        extras["per_world_path"] = {
            "agent_steps_per_s": job_rate(total_agents, 1, pw_ms), "ms_per_step": pw_ms,
            "launches_per_step": 2 * worlds.n_worlds}
        extras["speedup_vs_per_world_path"] = value / extras["per_world_path"]["agent_steps_per_s"]
        # batched precision path on the same worlds: FP16 reversed-Z keys, fused BF16 NCHW
        # normalised one-hot output (8 B/px), CUDA graph
        sim_p = Simulator(worlds, config_for(wl_rank, key_precision=1, output=1, autotune=1),
                          device=local)
        extras["precision_path"] = graph_rate(sim_p, worlds, wl_rank, 20)
        keep_sample("uniform_precision_bf16_f16key", sim_p, worlds, wl_rank)
        extras["precision_path"]["output"] = "bf16 NCHW one-hot (4 channels), f16 reversed-Z keys"
        extras["precision_path"]["speedup_vs_per_world_path"] = (
            extras["precision_path"]["agent_steps_per_s"] / extras["per_world_path"]["agent_steps_per_s"])
        sim_p.close()
        # the ray-traced backend on the same batch and outputs (step + trace per step)
        barrier()
        et = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        tr_steps = 10
        for k in range(2):
            sim.trace(out, depth)
        barrier()
        et[0].record(stream)
        for k in range(tr_steps):
            sim.trace(out, depth)
        et[1].record(stream)
        barrier()
        tr_ms = maxred(et[0].elapsed_time(et[1])) / tr_steps
        # step + trace replayed from one graph per step (gp_step_trace)
        for k in range(2):
            sim.step_trace(act, out, depth, stream=stream)
        barrier()
        et[0].record(stream)
        for k in range(tr_steps):
            sim.step_trace(act, out, depth, stream=stream)
        et[1].record(stream)
        barrier()
        st_ms = maxred(et[0].elapsed_time(et[1])) / tr_steps
        extras["ray_traced"] = {
            "trace_kernel_ms": tr_ms,
            "agent_steps_per_s_step_plus_trace": job_rate(total_agents, 1, st_ms),
            "ms_per_step_graph": st_ms,
            "render_gbs": algo_bytes / (tr_ms / 1e3) / 1e9,
            "render_frac_of_measured_hbm": algo_bytes / (tr_ms / 1e3) / 1e9 / peak,
            "note": "one ray per pixel: box slabs, lane-line and road plane hits via the grid"}
        # vectorized observations O_vec of every agent (16 agent, 32 road, 4 signal slots)
        obs = sim.observe_vec(stream=stream)
        barrier()
        eo = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        eo[0].record(stream)
        for k in range(10):
            sim.observe_vec(stream=stream, out=obs)
        eo[1].record(stream)
        barrier()
        extras["observe_vec"] = {"ms_per_call": maxred(eo[0].elapsed_time(eo[1])) / 10,
                                 "agents": n_agents, "slots_per_agent": [16, 32, 4],
                                 "note": "one warp per agent, nearest-K by warp sort/merge"}
        # the same batch with the reward terms and ego state computed in every step
        sim_w = Simulator(worlds, config_for(wl_rank, rewards=1, autotune=1), device=local)
        extras["with_rewards"] = graph_rate(sim_w, worlds, wl_rank, 20)
        extras["with_rewards"]["note"] = ("step computes the reward table's terms and the ego "
                                          "state for every agent (gp_get_rewards)")
        sim_w.close()
        # ragged batch at 256x144, precision path
        wl_r = rank_workload(wg.WORKLOADS["ragged_precision"], rank)
        worlds_r = wg.make_workload(wl_r)
        sim_r = Simulator(worlds_r, config_for(wl_r, autotune=1), device=local)
        extras["ragged_precision_256x144"] = graph_rate(sim_r, worlds_r, wl_r, 5)
        keep_sample("ragged_precision_256x144", sim_r, worlds_r, wl_r)
        extras["ragged_precision_256x144"]["workload"] = wl_r.name
        sim_r.close()
        # the ragged batch at 128x128 on the precision path (FP16 key, BF16 one-hot NCHW)
        wl_c = rank_workload(wg.WORKLOADS["ragged"], rank)
        worlds_c = wg.make_workload(wl_c)
        sim_c = Simulator(worlds_c, config_for(wl_c, autotune=1, key_precision=1, output=1),
                          device=local)
        extras["ragged_precision_128x128"] = graph_rate(sim_c, worlds_c, wl_c, 5)
        keep_sample("ragged_precision_128x128", sim_c, worlds_c, wl_c)
        extras["ragged_precision_128x128"]["workload"] = wl_c.name + ", f16 key, bf16 one-hot"
        sim_c.close()
        # the paper's observation rig: 4 cameras (0, +-60, 180 deg) at 434x252, shaded RGB
        wl_g = rank_workload(wg.WORKLOADS["paper_rig_434x252"], rank)
        worlds_g = wg.make_workload(wl_g)
        sim_g = Simulator(worlds_g, config_for(wl_g, autotune=1), device=local)
        extras["paper_rig_434x252_rgb"] = graph_rate(sim_g, worlds_g, wl_g, 5)
        extras["paper_rig_434x252_rgb"]["workload"] = wl_g.name
        extras["paper_rig_434x252_rgb"]["mpix_per_s"] = (
            extras["paper_rig_434x252_rgb"]["cameras"] * wl_g.width * wl_g.height /
            (extras["paper_rig_434x252_rgb"]["ms_per_step"] / 1e3) / 1e6)
        sim_g.close()

    if not args.no_sweep and not args.no_extras:
        # resolution sweep: 3 cameras (0, +-60 deg), 64 boxes, 1000 segments per world; the
        # batched precision path (f16 keys, bf16 one-hot) against the plain FP32 path (u8 class
        # + FP32 depth), square sizes 64..512, default launch shapes (no autotuning)
        wl_s0 = rank_workload(wg.WORKLOADS["sweep"], rank)
        worlds_s = wg.make_workload(wl_s0)
        sweep = {}
        for res in (64, 128, 256, 512):
            wl_s = dataclasses.replace(wl_s0, width=res, height=res)
            row = {}
            for path, kw, dep in (("plain_fp32_u8_class_f32_depth", dict(key_precision=0, output=0), True),
                                  ("precision_f16_key_bf16_onehot", dict(key_precision=1, output=1), False)):
                sim_s = Simulator(worlds_s, config_for(wl_s, **kw), device=local)
                r = graph_rate(sim_s, worlds_s, wl_s, 3, depth=dep)
                r["mpix_per_s"] = r["cameras"] * res * res / (r["ms_per_step"] / 1e3) / 1e6
                row[path] = r
                sim_s.close()
            row["precision_speedup"] = (row["precision_f16_key_bf16_onehot"]["agent_steps_per_s"] /
                                        row["plain_fp32_u8_class_f32_depth"]["agent_steps_per_s"])
            sweep["%dx%d" % (res, res)] = row
        extras["sweep_3cam"] = sweep

    # --- CPU leg: the oracle on this machine's host cores, after all GPU timing ---
    cpu = None
    if rank == 0:
        sampler = OracleSampler(wg.make_workload(wl_rank, n_worlds=min(worlds.n_worlds, 64)), wl_rank)
        rate, el, n = sampler.sample(args.cpu_seconds)
        sampler.close()
        cpu = {"value": rate, "unit": UNIT, "cores": sampler.cores, "kind": "oracle",
               "cpu": cpu_model(),
               "sample": "%d cameras (world step + one %dx%d render each) in %.1f s of wall time "
                         "on %d host cores, one process per core" % (
                             n, wl.width, wl.height, el, sampler.cores)}
        # the same oracle on the sampled GPU views of each configuration (from the GPU's state)
        acc = {k: accuracy_vs_oracle(v) for k, v in accuracy_samples.items()}
        if acc:
            extras["accuracy_vs_fp64_oracle"] = acc
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(wl, wl.n_worlds), "worlds_per_gpu": worlds.n_worlds,
                       "cameras_per_gpu": sim.n_views, "resolution": "%dx%d" % (wl.width, wl.height),
                       "output": "uint8 class + fp32 depth",
                       "renderer": "ray tracer (gp_step_trace)" if trace else "rasteriser",
                       "launch": "CUDA graph: step + %s" % ("trace" if trace else "render"),
                       "l2": "2x L2 buffer written between timed steps (outside the events); each "
                             "step also writes %.0f MB of images" % (out_bytes / 1e6),
                       "band_rows": sim.info.band_rows, "threads": sim.info.threads,
                       "tri_capacity": sim.info.tri_capacity, "blocks": sim.info.blocks,
                       "parallelism": "replicas" if world == 1 else "dp%d (independent worlds)" % world},
            "mpix_per_s": world * sim.n_views * px * args.steps / (total_ms / 1e3) / 1e6,
            "step_kernel_ms": stepk_ms, "render_kernel_ms": render_ms,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": 2 * args.steps, "clocks": clk.summary(),
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
