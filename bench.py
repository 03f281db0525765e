#!/usr/bin/env python
"""Benchmark: patch.atom Gibbs updates/s of BPFA dictionary learning on GB300.

Workload (one "step"): learn a dictionary from scratch on a 512x512 synthetic
STEM frame (two lattice grains with a 15 degree boundary, Poisson noise at
50 e-/px), 10% random mask, 10x10 patches at stride 1 (N = 253,009 patches,
P = 100), K = 128 atoms, 50 Gibbs iterations (code sweep, dictionary sweep,
pi / gamma draws), then the overlap-add reconstruction.  The frame is resident
in HBM; an L2 flush (256 MiB write) precedes every timed step.

value = N * K * iterations * steps / (sum of per-step CUDA-event times), over
all ranks (independent replicas, weak scaling).  ``e2e`` repeats the step
through the C ABI with pinned host buffers (frame copied in, reconstruction
copied out inside the timed region).  ``roofline`` reports the code-sweep
kernel against the SM issue ceiling; ``cpu_baseline`` times the FP64 oracle.

``--impl reference`` times the FP64 CPU oracle (the only reference for this
method) on the same workload: each step is one Gibbs iteration of a band of
frame rows, sized so the whole run ends within a few minutes.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(M=(512, 512), B=(10, 10), S=(1, 1), K=128, frac=0.10, grains=2, iters=50, seed=0)
WORKLOAD_NAME = ("stem512_k128: 512x512 two-grain synthetic STEM frame, 10% Bernoulli mask, "
                 "10x10 patches stride 1 (N=253009, P=100), K=128, 50 Gibbs iterations "
                 "(codes + dictionary + pi/gamma) from the prior, then overlap-add")
METRIC = "patch·atom Gibbs updates/s"
UNIT = "patch·atom updates/s"

# Algorithmic lane-operations of one code update:
#   2 |Omega_i| FMAs (masked norm + correlation), 75 fixed (Philox4x32-10:
#   60, log-odds / sigmoid / threshold: 15), 14 more when z = 1 (Box-Muller +
#   weight), |Omega_i| FMAs when the weight changes (rank-1 residual update).
# Plus patch extraction: |Omega_i| FMAs per non-zero stored weight where the
# sweep rebuilds the residual x_i - D w_i itself (stats.rebuild_observed).
OPS_FIXED, OPS_GAUSS = 75, 14
LANES_PER_SM = 128   # FP32 / INT32 lanes per SM (4 sub-partitions x 32)


def _frame():
    from paper_2311_15061_gb300 import synth
    x, clean = synth.stem_frame(WORKLOAD["M"], WORKLOAD["seed"], grains=WORKLOAD["grains"])
    mask = synth.random_mask(WORKLOAD["M"], WORKLOAD["frac"], WORKLOAD["seed"])
    return x, clean, mask


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _traffic_record(kernel_files):
    """dram bytes per launch of the code sweep from the committed ncu summary,
    valid only while the kernel sources are unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "sweep_kernel_stem512_k128_traffic.txt")
    try:
        kv = dict(line.split(":", 1) for line in open(path).read().splitlines() if ":" in line)
        blob = b"".join(open(os.path.join(ROOT, "paper_2311_15061_gb300", "csrc", f), "rb").read()
                        for f in kernel_files)
        digest = hashlib.sha256(blob).hexdigest()
        if kv.get("source_sha256", "").strip() != digest:
            return None
        return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region.

    Started before the warm-up and armed only once its first sample has
    arrived, so that nvidia-smi's own start-up never overlaps the timed steps.
    """

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []
        self.armed_at = None
        self._thread = None

    def start(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self

        def reader():
            for line in self.proc.stdout:
                self.lines.append(line)

        self._thread = threading.Thread(target=reader, daemon=True)
        self._thread.start()
        return self

    def wait_ready(self, timeout=30.0):
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.05)
        time.sleep(0.2)

    def arm(self):
        self.armed_at = len(self.lines)

    def stop(self):
        self.stopped_at = len(self.lines)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.out = "".join(self.lines[self.armed_at or 0:self.stopped_at])

    def summary(self):
        rows = []
        for line in getattr(self, "out", "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != self.gpu_index:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for _, _, r in rows for j in range(4) if r[j].lower() == "active"})
        busy = [r for r in rows if r[0] > 0.5 * r[1]] or rows
        return {"sm_mhz": statistics.median(r[0] for r in busy), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world):
    """The largest value of x over all ranks (the whole-job time is the slowest
    rank's); x itself when there is one rank.  Works with nccl (CUDA tensor)
    and gloo (CPU tensor)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_gpu(args):
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2311_15061_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2311_15061_gb300 import sensai

    x, clean, mask = _frame()
    w = WORKLOAD
    prm = sensai.make_params(w["M"], w["B"], w["S"], w["K"], seed=w["seed"] + rank)
    ctx = sensai.Context(prm, mask)
    N, K, iters = ctx.N, ctx.K, args.iters
    stream = torch.cuda.current_stream()
    frame = torch.from_numpy(x).cuda()
    out = torch.empty_like(frame)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    ctx.sensai_set_frame(frame, stream)

    def step():
        ctx.sensai_reset(stream)
        ctx.sensai_learn(None, iters, stream)
        ctx.sensai_reconstruct(out, stream)

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    gpu_index = int(vis) if vis.isdigit() else local
    clocks = ClockSampler(gpu_index).start()
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    clocks.wait_ready()
    if world > 1:
        torch.distributed.barrier()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = ctx.sensai_get_stats().kernel_launches
    ctx.sensai_profile(1)
    torch.cuda.synchronize()
    clocks.arm()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    time.sleep(0.15)
    clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    stats = ctx.sensai_get_stats()
    launches = stats.kernel_launches - launches0
    prof = ctx.sensai_profile_read()
    ctx.sensai_profile(0)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = max_over_ranks(sum(step_ms), world)
    updates = float(N) * K * iters * args.steps * world
    value = updates / (total_ms / 1e3)

    # roofline of the code sweep (dominant kernel)
    sweep_ms, sweep_n = prof["codes"]
    n_obs = ctx.sensai_get_stats().n_observed
    ops = (sweep_n * K * (2.0 * n_obs + OPS_FIXED * N) + float(stats.changed_observed)
           + OPS_GAUSS * float(stats.active_draws) + float(stats.rebuild_observed))
    peaks, peak_src = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = sms * LANES_PER_SM * sm_mhz * 1e6 / 1e12   # T lane-ops/s
    achieved = ops / sweep_n / (sweep_ms / sweep_n / 1e3) / 1e12
    traffic = _traffic_record(("sweep.cu", "sweep_block.cuh", "internal.cuh"))

    # end to end through the C ABI with pinned host buffers
    xh = torch.from_numpy(x).pin_memory()
    oh = torch.empty(x.shape, dtype=torch.float32).pin_memory()
    xh_np, oh_np = xh.numpy(), oh.numpy()
    e2e_steps = max(1, min(args.steps, 20))
    ctx.sensai_reset(stream)
    ctx.sensai_learn(xh_np, iters, stream)
    ctx.sensai_reconstruct(oh_np, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.sensai_reset(stream)
        ctx.sensai_learn(xh_np, iters, stream)
        ctx.sensai_reconstruct(oh_np, stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = float(N) * K * iters * e2e_steps * world / e2e_s

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "l2": "flushed before each step (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "patches": N, "atoms": K, "iterations": iters},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(x.nbytes),
                "d2h_bytes_per_step": int(x.nbytes), "steps": e2e_steps},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "kernel": "sweep_kernel (code sweep)", "achieved": achieved,
                     "peak": peak, "unit": "T lane-ops/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{sms} SMs x {LANES_PER_SM} lanes x {sm_mhz:.0f} MHz ({peak_src} max SM clock)",
                     "ms_per_launch": sweep_ms / sweep_n, "launches": sweep_n},
        "phases_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "wall_s": wall,
        "clocks": clocks.summary(),
    }
    line["posterior_mean"] = posterior_mean_psnr(ctx, clean, iters, stream=stream)
    if not args.no_serving:
        line["serving"] = run_serving(ctx, dict(B=w["B"], S=w["S"], K=w["K"], seed=w["seed"] + rank))
    if not args.no_video:
        line["video3d"] = run_video3d()
    if not args.no_batch:
        line["batch64"] = run_batch64()
    if not args.no_precision and world == 1:
        line["precision"] = run_precision()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


SERVE = dict(frames=300, sizes=((256, 256), (512, 512), (1024, 1024)), streams=4, rate_hz=20.0,
             frac=(0.05, 0.20), sweeps=3, slots=8, closed_1024=48, overload_hz=100.0, overload_frames=400,
             overload_budget_1024=4, psnr_1024=4, seed=7)

_MASK64 = (1 << 64) - 1


def _splitmix64(x):
    """SplitMix64's finaliser (Steele, Lea, Flood 2014): the serving engine keys
    each frame's draws with h(h(h(seed) ^ stream) ^ frame)."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def _serving_requests(cfg, rate_hz, frames, seed):
    """The live-feed workload: frames of mixed sizes from a drifting-lattice
    pool, each with its own random or line-hop mask (5-20%), arriving as four
    Poisson streams."""
    from paper_2311_15061_gb300 import synth
    rng = np.random.default_rng(seed)
    pool = {shp: [synth.stem_frame(shp, cfg["seed"] + j, drift=(0.0, 0.3 * j)) for j in range(3)]
            for shp in cfg["sizes"]}
    reqs = []
    t_stream = np.zeros(cfg["streams"])
    for n in range(frames):
        sid = n % cfg["streams"]
        t_stream[sid] += rng.exponential(1.0 / rate_hz)
        shp = cfg["sizes"][int(rng.integers(0, len(cfg["sizes"])))]
        frac = float(rng.uniform(*cfg["frac"]))
        mask = (synth.random_mask(shp, frac, seed + n) if n % 2 == 0
                else synth.line_hop_mask(shp, frac, seed + n))
        reqs.append(dict(t=float(t_stream[sid]), stream=sid, frame_id=n, shape=shp,
                         x=pool[shp][n % 3][0], mask=mask))
    reqs.sort(key=lambda r: r["t"])
    return reqs, pool


def _open_loop(ctx, reqs, cfg, id_base):
    """Submits each request at its arrival time; returns the latencies (ms,
    submission to completion callback), achieved frames/s and per-size stats."""
    import threading
    lock = threading.Lock()
    finished = {}

    def on_done(fid, status, out):
        with lock:
            finished[fid] = (time.perf_counter(), status)

    submitted = {}
    t0 = time.perf_counter()
    for r in reqs:
        delay = t0 + r["t"] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        fid = id_base + r["frame_id"]
        submitted[fid] = (time.perf_counter(), r["shape"])
        ctx.sensai_submit_frame(r["stream"], fid, r["x"], r["mask"], cfg["sweeps"], done=on_done)
    ctx.sensai_serve_drain()
    t_end = max(v[0] for v in finished.values())
    lat = {fid: 1e3 * (finished[fid][0] - submitted[fid][0]) for fid in submitted}
    all_lat = np.array(list(lat.values()))
    by_size = {}
    for shp in cfg["sizes"]:
        v = np.array([lat[f] for f, (_, s_) in submitted.items() if s_ == shp])
        if len(v):
            by_size[f"{shp[0]}x{shp[1]}"] = {"frames": int(len(v)), "p50_ms": float(np.percentile(v, 50)),
                                             "p99_ms": float(np.percentile(v, 99))}
    return {"frames": len(reqs), "fps": len(reqs) / (t_end - t0), "p50_ms": float(np.percentile(all_lat, 50)),
            "p99_ms": float(np.percentile(all_lat, 99)), "by_size": by_size,
            "all_ok": all(finished[f][1] == 0 for f in submitted)}


def _serve_psnr(ctx, cfg, params, state):
    """PSNR of served 1024^2 frames against the clean frame, and whether each
    equals sensai_inpaint on a context keyed by the frame's own seed."""
    from paper_2311_15061_gb300 import sensai, synth
    import threading
    big = cfg["sizes"][-1]
    res = []
    done = threading.Event()
    for j in range(cfg["psnr_1024"]):
        x, clean = synth.stem_frame(big, cfg["seed"] + 100 + j, drift=(0.0, 0.3 * j))
        m = synth.random_mask(big, 0.1, 900 + j)
        done.clear()
        out = ctx.sensai_submit_frame(2, 30_000_000 + j, x, m, cfg["sweeps"], done=lambda f, st, o: done.set())
        ctx.sensai_serve_drain()
        fseed = _splitmix64(_splitmix64(_splitmix64(params["seed"]) ^ 2) ^ (30_000_000 + j))
        c2 = sensai.Context(sensai.make_params(big, params["B"], params["S"], params["K"], seed=fseed), m)
        c2.sensai_set_state(D=state["D"], pi=state["pi"], gamma_s=state["gamma_s"], gamma_eps=state["gamma_eps"],
                            iter=state["iter"])
        ref = np.empty(big, np.float32)
        c2.sensai_inpaint(x, cfg["sweeps"], ref)
        c2.close()

        def psnr(a, b):
            mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
            return 10.0 * np.log10(1.0 / mse)
        res.append({"psnr_served_vs_clean_db": psnr(out, clean), "psnr_noisy_frame_vs_clean_db": psnr(x, clean),
                    "equals_inpaint": bool(np.array_equal(out, ref))})
    return {"frames": len(res), "mask": "10% Bernoulli", "mean_psnr_served_vs_clean_db":
            float(np.mean([r["psnr_served_vs_clean_db"] for r in res])),
            "mean_psnr_noisy_frame_vs_clean_db": float(np.mean([r["psnr_noisy_frame_vs_clean_db"] for r in res])),
            "all_equal_inpaint": all(r["equals_inpaint"] for r in res)}


def run_serving(ctx, params, cfg=SERVE):
    """Live serving: an open-loop Poisson load, a closed loop at 1024^2 with
    every slot busy (per-frame latency), an offered load above capacity under
    a memory budget, and the PSNR of served frames."""
    import threading
    from paper_2311_15061_gb300 import synth
    state = ctx.sensai_get_state()
    big = cfg["sizes"][-1]
    ctx.sensai_serve_start(slots=cfg["slots"], max_pixels=big[0] * big[1], max_observed=64)
    # warm-up: one frame of each size
    for j, shp in enumerate(cfg["sizes"]):
        x, _ = synth.stem_frame(shp, cfg["seed"] + 50 + j)
        ctx.sensai_submit_frame(9, 10_000_000 + j, x, synth.random_mask(shp, 0.1, j), cfg["sweeps"])
    ctx.sensai_serve_drain()

    reqs, pool = _serving_requests(cfg, cfg["rate_hz"], cfg["frames"], cfg["seed"])
    mixed = _open_loop(ctx, reqs, cfg, 0)
    mixed["offered_hz"] = cfg["rate_hz"] * cfg["streams"]

    # closed loop at 1024^2: a new frame as soon as one completes, `slots` in flight
    lock = threading.Lock()
    cv = threading.Condition(lock)
    t_done = {}
    masks = [synth.random_mask(big, 0.1, 500 + j) for j in range(8)]
    frames_big = [v[0] for v in pool[big]]

    def on_done(fid, status, out):
        with cv:
            t_done[fid] = (time.perf_counter(), status)
            cv.notify()

    t_sub = {}
    n = cfg["closed_1024"]
    t1 = time.perf_counter()
    for j in range(n):
        with cv:
            while j - len(t_done) >= cfg["slots"]:
                cv.wait()
        t_sub[20_000_000 + j] = time.perf_counter()
        ctx.sensai_submit_frame(j % cfg["streams"], 20_000_000 + j, frames_big[j % 3], masks[j % 8], cfg["sweeps"],
                                done=on_done)
    ctx.sensai_serve_drain()
    t2 = max(v[0] for v in t_done.values())
    lat = np.array([1e3 * (t_done[f][0] - t_sub[f]) for f in t_sub])
    closed = {"frames": n, "in_flight": cfg["slots"], "fps": n / (t2 - t1),
              "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
              "all_ok": all(v[1] == 0 for v in t_done.values())}
    psnr = _serve_psnr(ctx, cfg, params, state)
    ctx.sensai_serve_stop()

    # above capacity: 4 streams x overload_hz, memory budget of a few 1024^2 frames
    ctx.sensai_serve_start(slots=cfg["slots"], max_pixels=big[0] * big[1], max_observed=64,
                           memory_budget=_frame_footprint(params, big) * cfg["overload_budget_1024"])
    for j, shp in enumerate(cfg["sizes"]):
        x, _ = synth.stem_frame(shp, cfg["seed"] + 60 + j)
        ctx.sensai_submit_frame(9, 11_000_000 + j, x, synth.random_mask(shp, 0.1, j), cfg["sweeps"])
    ctx.sensai_serve_drain()
    oreqs, _ = _serving_requests(cfg, cfg["overload_hz"], cfg["overload_frames"], cfg["seed"] + 1)
    over = _open_loop(ctx, oreqs, cfg, 40_000_000)
    over["offered_hz"] = cfg["overload_hz"] * cfg["streams"]
    over["memory_budget_bytes"] = _frame_footprint(params, big) * cfg["overload_budget_1024"]
    ctx.sensai_serve_stop()
    return {"workload": ("frames of 256^2/512^2/1024^2, random or line-hop masks 5-20%, 3 code sweeps + pi/gamma "
                         "draws per frame, K=128 10x10 dictionary transferred from the learning step, 8 slots"),
            "mixed_4x20hz": mixed, "closed_loop_1024": closed, "overload": over, "psnr_1024": psnr}


def _frame_footprint(params, shape):
    """Device bytes the serving engine charges a frame of this shape (the
    engine's own accounting is in csrc/serve.cu; this mirrors its terms:
    frame, mask, output, per-patch tables, weights and activity bits)."""
    P = int(np.prod(params["B"]))
    N = int(np.prod([(m - b) // s + 1 for m, b, s in zip(shape, params["B"], params["S"])]))
    K = params["K"]
    npx = int(np.prod(shape))
    NW = (N + 31) // 32
    KB = (K + 7) // 8
    max_observed = 64
    return int(8 * npx + npx + 4 * ((npx + 31) // 32) + 2 * N * (1 + max_observed) + 4 * KB * 8 * NW * 32
               + 4 * K * NW + 32 * NW + 4 * P * N)


VIDEO = dict(M=(32, 256, 256), B=(4, 8, 8), S=(2, 1, 1), K=256, frac=0.15, iters=30, seed=0)


def run_video3d(cfg=VIDEO):
    """3-D video cube: 32 frames of 256x256 (drifting lattice), 15% Bernoulli
    mask, 4x8x8 patches at stride (2, 1, 1) (N = 930,015, P = 256), K = 256,
    30 Gibbs iterations from the prior.  The dictionary (257 KB in FP32)
    does not fit in shared memory, so the code sweep streams it in slices.
    Timed once after a warm-up call, frame resident on the device."""
    import torch
    from paper_2311_15061_gb300 import sensai, synth
    x, clean = synth.stem_volume(cfg["M"], cfg["seed"])
    mask = synth.random_mask(cfg["M"], cfg["frac"], cfg["seed"])
    ctx = sensai.Context(sensai.make_params(cfg["M"], cfg["B"], cfg["S"], cfg["K"], seed=cfg["seed"]), mask)
    stream = torch.cuda.current_stream()
    frame = torch.from_numpy(x).cuda()
    out = torch.empty_like(frame)
    ctx.sensai_set_frame(frame, stream)
    ctx.sensai_learn(None, 2, stream)         # warm-up
    ctx.sensai_reset(stream)
    torch.cuda.synchronize()
    ctx.sensai_profile(1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.sensai_learn(None, cfg["iters"], stream)
    ctx.sensai_reconstruct(out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = ctx.sensai_profile_read()
    ctx.sensai_profile(0)
    st = ctx.sensai_get_stats()
    rec = out.cpu().numpy().astype(np.float64)
    psnr = float(10 * np.log10(1.0 / np.mean((rec - clean) ** 2)))
    res = {"workload": ("video3d_k256: 32x256x256 drifting-lattice video, 15% Bernoulli mask, 4x8x8 patches "
                        "stride (2,1,1) (N=930015, P=256), K=256, 30 Gibbs iterations from the prior, then "
                        "overlap-add"),
           "value": float(st.n_patches) * cfg["K"] * cfg["iters"] / (ms / 1e3), "unit": UNIT,
           "ms_per_iteration": ms / cfg["iters"],
           "phases_ms_per_iteration": {k: v[0] / cfg["iters"] for k, v in prof.items()},
           "slice_atoms": st.slice_atoms, "slices": st.slices, "max_observed": st.max_observed,
           "psnr_db_vs_clean": psnr,
           "posterior_mean": posterior_mean_psnr(ctx, clean, cfg["iters"], stream=stream)}
    ctx.close()
    return res


PRECISION_ITERS = 50
MEAN_LAST = 10


def posterior_mean_psnr(ctx, clean, iters, last=MEAN_LAST, stream=None):
    """From the prior, iters Gibbs iterations with the overlap-add
    reconstructions of the last `last` accumulated on the device: PSNR
    against the clean frame of the final sample and of the mean of the last
    `last` samples (the posterior-mean estimate)."""
    def psnr(a):
        return float(10 * np.log10(1.0 / np.mean((a.astype(np.float64) - clean) ** 2)))
    last = max(1, min(last, iters))
    ctx.sensai_reset(stream)
    ctx.sensai_learn(None, iters - last, stream)
    ctx.sensai_mean_reset(stream)
    for _ in range(last):
        ctx.sensai_learn(None, 1, stream)
        ctx.sensai_mean_add(stream)
    final = ctx.sensai_reconstruct(None, stream)
    mean = ctx.sensai_mean_read(None, stream)
    return {"iterations": iters, "last_samples": last, "psnr_final_sample_db": psnr(final),
            "psnr_mean_of_last_db": psnr(mean)}


def run_precision():
    """The dictionary draw's three forms on the 512x512, K = 128 workload:
    the residual form (FP32, the default), the dense-statistics form with
    FP32-level Grams (TF32 head/tail split on the tensor cores) and with
    TF32-level Grams.  Per form: the dictionary phase and whole iteration
    times over 50 Gibbs iterations from the prior, the PSNR of the final
    reconstruction, and -- from one shared state (the residual form's after
    10 iterations) -- the largest per-atom relative difference of one
    dictionary draw from the residual form's draw.  The errors against the
    FP64 oracle are measured by the parity tests."""
    import torch
    from paper_2311_15061_gb300 import sensai
    x, clean, mask = _frame()
    w = WORKLOAD
    stream = torch.cuda.current_stream()
    frame = torch.from_numpy(x).cuda()
    forms = {"residual_fp32": 0, "dense_fp32_split": sensai.SENSAI_FLAG_DENSE_STATISTICS,
             "dense_tf32": sensai.SENSAI_FLAG_TF32_STATISTICS}
    ref = sensai.Context(sensai.make_params(w["M"], w["B"], w["S"], w["K"], seed=w["seed"]), mask)
    ref.sensai_learn(x, 10)
    state = ref.sensai_get_state()
    ref.sensai_draw_dictionary()
    d_ref = ref.sensai_get_dictionary().astype(np.float64)
    ref.close()
    res = {"workload": WORKLOAD_NAME, "iterations": PRECISION_ITERS, "forms": {}}
    for name, flags in forms.items():
        ctx = sensai.Context(sensai.make_params(w["M"], w["B"], w["S"], w["K"], seed=w["seed"], flags=flags), mask)
        ctx.sensai_set_frame(frame, stream)
        ctx.sensai_learn(None, 3, stream)   # warm-up
        ctx.sensai_reset(stream)
        torch.cuda.synchronize()
        ctx.sensai_profile(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.sensai_learn(None, PRECISION_ITERS, stream)
        e1.record(stream)
        out = ctx.sensai_reconstruct()
        torch.cuda.synchronize()
        prof = ctx.sensai_profile_read()
        ctx.sensai_profile(0)
        psnr = float(10 * np.log10(1.0 / np.mean((out.astype(np.float64) - clean) ** 2)))
        ctx.sensai_set_state(**state)
        ctx.sensai_draw_dictionary()
        d = ctx.sensai_get_dictionary().astype(np.float64)
        diff = np.linalg.norm(d - d_ref, axis=1) / np.maximum(np.linalg.norm(d_ref, axis=1), 1e-30)
        res["forms"][name] = {
            "ms_per_iteration": e0.elapsed_time(e1) / PRECISION_ITERS,
            "dictionary_ms_per_iteration": prof["dictionary"][0] / PRECISION_ITERS,
            "psnr_db_vs_clean": psnr,
            "dictionary_draw_max_rel_diff_vs_residual_fp32": float(diff.max()),
        }
        ctx.close()
    return res


BATCH = dict(sizes=(64, 96, 128, 192, 256, 384, 512), per_size=8, cubes=8, cube_shape=(128, 128, 512),
             cube_B=(4, 4, 32), cube_S=(1, 1, 32), Ks=(64, 128, 256), frac2d=(0.05, 0.30),
             frac_cube=(0.05, 0.30), iters=20, seed=11)


def _batch_instances(cfg=BATCH):
    """The heterogeneous set: 2-D frames of every size with 8x8 patches and
    spectrum-image cubes with 4x4x32 patches at stride (1, 1, 32), K cycling
    through 64 / 128 / 256, Bernoulli masks at per-instance fractions."""
    from paper_2311_15061_gb300 import synth
    rng = np.random.default_rng(cfg["seed"])
    inst = []
    n = 0
    for sz in cfg["sizes"]:
        for j in range(cfg["per_size"]):
            x, _ = synth.stem_frame((sz, sz), cfg["seed"] + n, grains=1 + (n % 2))
            frac = float(rng.uniform(*cfg["frac2d"]))
            inst.append(dict(M=(sz, sz), B=(8, 8), S=(1, 1), K=cfg["Ks"][n % 3], x=x,
                             mask=synth.random_mask((sz, sz), frac, cfg["seed"] + n)))
            n += 1
    cubes = [synth.spectrum_cube(cfg["cube_shape"], cfg["seed"] + 100 + j)[0] for j in range(cfg["cubes"] // 2)]
    for j in range(cfg["cubes"]):
        frac = float(rng.uniform(*cfg["frac_cube"]))
        inst.append(dict(M=cfg["cube_shape"], B=cfg["cube_B"], S=cfg["cube_S"], K=cfg["Ks"][n % 3],
                         x=cubes[j % len(cubes)], mask=synth.random_mask(cfg["cube_shape"], frac, cfg["seed"] + n)))
        n += 1
    return inst


def run_batch64(cfg=BATCH):
    """64 independent instances learned together (sensai_batch_*): one graph
    replay per Gibbs iteration after autotuning, against the same 20
    iterations run instance after instance with sensai_learn."""
    import torch
    from paper_2311_15061_gb300 import sensai
    inst = _batch_instances(cfg)
    ctxs = []
    for j, c in enumerate(inst):
        p = sensai.make_params(c["M"], c["B"], c["S"], c["K"], seed=cfg["seed"] + j,
                               flags=sensai.SENSAI_FLAG_CHAIN_DICTIONARY)
        ctx = sensai.Context(p, c["mask"])
        ctx.sensai_set_frame(c["x"])
        ctxs.append(ctx)
    updates = float(sum(ctx.N * ctx.K for ctx in ctxs)) * cfg["iters"]
    stream = torch.cuda.current_stream()
    batch = sensai.Batch(ctxs)
    divisor = batch.sensai_batch_tune(1, stream)
    for ctx in ctxs:
        ctx.sensai_reset(stream)
    batch.sensai_batch_learn(1, stream)            # the tuned graph's capture, off the clock
    for ctx in ctxs:
        ctx.sensai_reset(stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    batch.sensai_batch_learn(cfg["iters"], stream)
    e1.record(stream)
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1)
    batch.close()
    for ctx in ctxs:
        ctx.sensai_reset(stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for ctx in ctxs:
        ctx.sensai_learn(None, cfg["iters"], stream)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    res = {"workload": ("batch64: 56 synthetic STEM frames 64^2..512^2 (8x8 patches, masks 5-30%) + 8 spectrum "
                        "cubes 128x128x512 (4x4x32 patches stride (1,1,32), masks 5-30%), K in {64,128,256}, "
                        "20 Gibbs iterations from the prior"),
           "instances": len(ctxs), "patch_atom_updates": updates,
           "value": updates / (batched_ms / 1e3), "unit": UNIT, "ms": batched_ms,
           "sequential_value": updates / (seq_ms / 1e3), "sequential_ms": seq_ms,
           "speedup_vs_sequential": seq_ms / batched_ms, "tuned_sweep_grid_divisor": divisor}
    for ctx in ctxs:
        ctx.close()
    return res


def _oracle_band(rows):
    """The workload restricted to the first ``rows`` frame rows."""
    import oracle as O
    x, clean, mask = _frame()
    w = WORKLOAD
    xs, ms = np.ascontiguousarray(x[:rows]), np.ascontiguousarray(mask[:rows])
    prm = O.params((rows, w["M"][1]), w["B"], w["S"], w["K"], seed=w["seed"])
    return O, prm, xs, ms


def _oracle_iteration(rows, iters=1):
    O, prm, xs, ms = _oracle_band(rows)
    st = O.State(prm)
    t0 = time.perf_counter()
    O.learn(st, xs, ms, iters)
    dt = time.perf_counter() - t0
    return O.num_patches(prm) * prm.K * iters, dt, O.num_threads()


def cpu_baseline():
    rows = WORKLOAD["M"][0]
    upd, dt, cores = _oracle_iteration(rows, 1)
    return {"value": upd / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"1 full Gibbs iteration (codes + dictionary + pi/gamma) of the full 512x512 "
                      f"K=128 workload from the prior, {dt:.1f} s"}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    budget_s = 150.0
    # calibrate on a small band, then size the per-step band to the budget
    upd, dt, cores = _oracle_iteration(24, 1)
    per_row_s = dt / 24.0
    steps_total = args.steps + args.warmup
    rows = int(max(12, min(WORKLOAD["M"][0], budget_s / steps_total / per_row_s)))
    for _ in range(args.warmup):
        _oracle_iteration(rows, 1)
    total_upd, total_s = 0.0, 0.0
    for _ in range(args.steps):
        u, d, cores = _oracle_iteration(rows, 1)
        total_upd += u
        total_s += d
    value = total_upd / total_s
    sample = (f"per step: 1 Gibbs iteration (codes + dictionary + pi/gamma) of the first {rows} "
              f"of 512 frame rows of the workload (same patch size, K, mask density)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_NAME},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["sensai", "reference"], default="sensai")
    ap.add_argument("--iters", type=int, default=WORKLOAD["iters"],
                    help="Gibbs iterations per step (50 is the workload; fewer only for profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the live-serving measurement")
    ap.add_argument("--no-video", action="store_true", help="skip the 3-D video measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-instances measurement")
    ap.add_argument("--no-precision", action="store_true", help="skip the dictionary-form comparison")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
