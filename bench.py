"""Throughput benchmark: Siddon DRR forward + pose gradient on one GB300.

Workload (the headline configuration): a 512x512x133 chest-CT-shaped volume
(seeded int16 HU phantom mapped to FP32 attenuation, spacing 0.703 x 0.703 x
2.5 mm), a 200x200 detector at 1.4 mm, SDR 510 mm, a batch of 16 random poses.
One step = the whole hot path for that batch: pose setup, the fused Siddon
forward with per-ray pose Jacobian (DRR + dE/d eta), and the deterministic
reduction of a seeded upstream gradient to dL/d pose.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the host cores instead, on a bounded sample of the same workload.
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

METRIC = "Gray-s fwd & fwd+pose-grad at 512x512x133 CT, 200x200 det; served p50/p99 ms"
UNIT = "Grays/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        # the raw samples; their summary goes into the JSON line
        self.path = os.path.join(os.environ.get("DRR_BENCH_LOG_DIR", tempfile.gettempdir()),
                                 f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_batch(cfg, rank):
    """The poses and upstream gradient one rank renders.  Poses are independent
    problems, so N ranks each take their own batch of cfg["batch"] poses (weak
    scaling, no data-path collective); rank 0's batch is the single-GPU one."""
    from paper_2208_12737_gb300 import inputs
    det = cfg["detector"]
    poses = inputs.random_poses(cfg["batch"], seed=cfg["pose_seed"] + 1000 * rank)
    g = inputs.upstream_grad((cfg["batch"], det.height, det.width), seed=3 + 1000 * rank)
    return poses, g


def max_over_ranks(values, dist=None, device=None):
    """Element-wise maximum of per-rank timings (the slowest rank sets the job time)."""
    import torch
    t = torch.tensor([float(x) for x in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_throughput(world, rays_per_rank, ms):
    """Whole-job rays per second (G rays/s) when every rank renders rays_per_rank in ms."""
    return world * rays_per_rank / (ms * 1e-3) / 1e9


def timed_steps(fn, k, before=None, clock="cuda"):
    """Run fn k times and return the duration of each call in ms.  clock="cuda":
    CUDA events recorded on the current stream around each call (after an
    untimed `before()`, e.g. an L2 flush); clock="host": perf_counter around
    each call (the CPU stand-in used by the multi-process tests)."""
    if clock == "host":
        out = []
        for i in range(k):
            if before is not None:
                before(i)
            t0 = time.perf_counter()
            fn()
            out.append((time.perf_counter() - t0) * 1e3)
        return out
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
    for i in range(k):
        if before is not None:
            before(i)
        starts[i].record()
        fn()
        ends[i].record()
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def job_timing(world, rays_per_rank, per_rank_ms, dist=None, device=None):
    """Whole-job figures from each rank's mean step times (a list, one entry per
    timed quantity): the slowest rank sets every time, and the throughput counts
    the rays of all ranks.  Returns (max-over-ranks ms list, throughput list)."""
    ms = max_over_ranks([statistics.mean(x) for x in per_rank_ms], dist, device)
    return ms, [job_throughput(world, rays_per_rank, m) for m in ms]


def resolve_world(gpus, env=None):
    """(rank, world, local_rank) of this process.  A run with --gpus N > 1 must be
    launched one process per GPU (torchrun --nproc-per-node N), which sets
    WORLD_SIZE = N; anything else is an error, so a multi-GPU run can never
    print a one-rank number."""
    env = os.environ if env is None else env
    if gpus < 1:
        raise SystemExit("bench.py: --gpus must be >= 1")
    if "WORLD_SIZE" in env:
        world = int(env["WORLD_SIZE"])
        if world != gpus:
            raise SystemExit(f"bench.py: --gpus {gpus} but WORLD_SIZE={world}: launch one process per GPU "
                             f"with torchrun --nproc-per-node {gpus}")
    elif gpus > 1:
        raise SystemExit(f"bench.py: --gpus {gpus} needs one process per GPU: run it as "
                         f"python -m torch.distributed.run --nproc-per-node {gpus} --master-addr 127.0.0.1 "
                         f"bench.py --gpus {gpus} ...")
    else:
        world = 1
    return int(env.get("RANK", "0")), world, int(env.get("LOCAL_RANK", "0"))


def kernel_source_hash():
    """sha256 of the walk kernels' sources: a stored ncu traffic figure applies only to this source."""
    import hashlib
    h = hashlib.sha256()
    for f in ("drr_kernels.cu", "drr_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2208_12737_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_value(key, kernel="siddon_fwd_jac"):
    """A per-launch figure (`key: N source_sha256: H`) from the committed ncu summary
    of `kernel`, if it was taken on the current kernel source; else None."""
    import glob
    import re
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{kernel}__*.md"))):
        with open(path) as f:
            text = f.read()
        m = re.search(key + r":\s*(\d+)\s+source_sha256:\s*([0-9a-f]{64})", text)
        if m and m.group(2) == kernel_source_hash():
            return int(m.group(1))
    return None


def profiled_traffic(kernel="siddon_fwd_jac"):
    """DRAM bytes per launch of `kernel` (ncu), for the current kernel source; else None."""
    return profiled_value("traffic_bytes_per_launch", kernel)


def issue_roofline(kernel_ms, sm_max_mhz):
    inst = profiled_value("warp_instructions_per_launch")
    peak = 4 * 152 * sm_max_mhz * 1e6 / 1e9  # G warp-instructions/s
    if inst is None:
        return {"achieved_ginst_s": None, "peak_ginst_s": peak, "frac": None}
    ach = inst / (kernel_ms * 1e-3) / 1e9
    return {"achieved_ginst_s": ach, "peak_ginst_s": peak, "frac": ach / peak, "inst_per_launch": inst}


def workload_inputs(rank=0):
    from paper_2208_12737_gb300 import inputs
    cfg = inputs.CT
    hu = inputs.ct_volume_hu()
    poses, g = rank_batch(cfg, rank)
    return cfg, hu, poses, g


_ORACLE_CTX = {}


def cpu_oracle_sample(cfg, hu, poses, seconds_target=10.0, threads=0):
    """Time the FP64 oracle (forward + per-ray pose Jacobian) on a bounded pixel sample.
    The oracle's volume and a calibration of its ray rate are prepared once per workload."""
    import oracle
    from paper_2208_12737_gb300 import inputs
    d = cfg["detector"]
    cores = threads if threads > 0 else (os.cpu_count() or 1)
    key = (cfg["name"], id(hu), cores)
    if key not in _ORACLE_CTX:
        f32 = lambda x: float(np.float32(x))
        mu = oracle.hu_to_mu(hu, inputs.MU_WATER).astype(np.float32)
        ov = oracle.Volume(mu, tuple(f32(s) for s in cfg["spacing"]))
        det = (f32(d.sdr), d.height, d.width, f32(d.delta_h), f32(d.delta_w))
        # calibrate on a small sample, then size each timed sample to about seconds_target
        npix = 64
        cal = np.random.default_rng(122).integers(0, d.height * d.width, npix)
        t0 = time.perf_counter()
        oracle.render(ov, det, poses, pixels=cal, jacobian=True, threads=cores)
        dt = max(time.perf_counter() - t0, 1e-3)
        _ORACLE_CTX[key] = (ov, det, poses.shape[0] * npix / dt, np.random.default_rng(123))
    ov, det, rate, rng = _ORACLE_CTX[key]
    npix = int(min(d.height * d.width, max(64, rate * seconds_target / poses.shape[0])))
    pix = rng.choice(d.height * d.width, size=npix, replace=False)
    t0 = time.perf_counter()
    oracle.render(ov, det, poses, pixels=pix, jacobian=True, threads=cores)
    dt = time.perf_counter() - t0
    rays = poses.shape[0] * npix
    return {"value": rays / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{npix} random pixels x {poses.shape[0]} poses of the 512x512x133/200x200 workload "
                      f"(fwd + per-ray pose Jacobian, FP64), {dt:.1f} s"}, dt, rays


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    cfg, hu, poses, _ = workload_inputs()
    per = []
    base = None
    for i in range(args.warmup + args.steps):
        # each step a bounded sample: the whole run is about 90 s of oracle work for any K and W
        cb, dt, rays = cpu_oracle_sample(cfg, hu, poses, seconds_target=max(0.02, 90.0 / (args.steps + args.warmup)))
        if i >= args.warmup:
            per.append(cb["value"])
            base = cb
    value = statistics.median(per)
    base["value"] = value
    rays_per_step = cfg["batch"] * cfg["detector"].height * cfg["detector"].width
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rays_per_step / (value * 1e9) * 1e3,
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "volume": "512x512x133 HU->FP32", "detector": "200x200 @1.4mm",
                       "batch": cfg["batch"], "sample": base["sample"]},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serving_volumes(drr, hu133):
    """The serving workload's 8 resident volumes: {128^3 @2 mm, 256^3 @1 mm, 512x512x133,
    512x512x300} x {FP32, BF16}."""
    from paper_2208_12737_gb300 import inputs
    specs = [
        ("128^3", lambda: (inputs.ellipsoid_phantom((128, 128, 128), (2.0, 2.0, 2.0), seed=81,
                                                    semi_range=(10, 60), density_range=(0.0, 0.01)), False),
         (2.0, 2.0, 2.0)),
        ("256^3", lambda: (inputs.ellipsoid_phantom((256, 256, 256), (1.0, 1.0, 1.0), seed=82,
                                                    semi_range=(10, 60), density_range=(0.0, 0.01)), False),
         (1.0, 1.0, 1.0)),
        ("512x512x133", lambda: (hu133, True), (0.703, 0.703, 2.5)),
        ("512x512x300", lambda: (inputs.ct_phantom_hu((300, 512, 512), (0.703, 0.703, 1.1), seed=83), True),
         (0.703, 0.703, 1.1)),
    ]
    vols = []
    for name, make, sp in specs:
        data, hu = make()
        for storage in ("f32", "bf16"):
            vols.append((f"{name}/{storage}", drr.Volume(data, sp, hu=hu, storage=storage)))
    return vols


SERVE_TICK_WORK = 1 << 30  # ray-planes admitted into one tick (about 0.5-0.8 ms of walk)


def serve_bench(drr, hu133, seconds=2.0, seed=8, sat_requests=2000, loads=(0.25, 0.5, 0.8, 0.95),
                max_tick_work=SERVE_TICK_WORK, plain=True, vols=None, tick_depth=0):
    """Served latency: saturation throughput, then Poisson arrivals at fractions of it;
    beside it the plain FP32 comparison server, measured the same way."""
    import threading
    from paper_2208_12737_gb300 import inputs
    vols = vols or serving_volumes(drr, hu133)
    rng = np.random.default_rng(seed)
    grads = {}

    # The client's result buffers: a few per detector size, allocated and touched
    # once and reused round robin, as a client that keeps its buffers would (fresh
    # arrays per request make the server's result copy take their page faults)
    out_pool, out_next = {}, {}

    def out_for(n):
        if n not in out_pool:
            out_pool[n] = [np.zeros((1, n, n), np.float32) for _ in range(4)]
            out_next[n] = 0
        out_next[n] = (out_next[n] + 1) % 4
        return out_pool[n][out_next[n]]

    def make_req():
        name, v = vols[int(rng.integers(len(vols)))]
        n = int(rng.integers(128, 513))
        det = inputs.Detector(510.0, n, n, 280.0 / n, 280.0 / n)
        pose = inputs.random_poses(1, seed=int(rng.integers(1 << 30)))
        g = None
        if rng.uniform() < 0.5:
            if n not in grads:
                grads[n] = inputs.upstream_grad((1, n, n), seed=n)
            g = grads[n]
        return v, det, pose, g, out_for(n)

    def submit(srv, r):
        v, det, pose, g, out = r
        return srv.submit(v, det, pose, g, out=out)

    def drain(tickets, lat):
        for t in tickets:
            t.wait(120000)
            lat.append(t.result.latency_ms)

    def new_server(plain_mode=False):
        if plain_mode:
            return drr.Server(device_budget=2 << 30, max_inflight=64, plain_fp32_baseline=True)
        return drr.Server(device_budget=2 << 30, max_inflight=64, use_cuda_graph=True, max_tick_work=max_tick_work,
                          tick_depth=tick_depth)

    def saturation(reqs, plain_mode=False):
        """Everything queued at once; after one untimed pass, the median of three timed passes."""
        srv = new_server(plain_mode)
        for r in reqs[:32]:
            submit(srv, r).wait(120000)
        drain([submit(srv, r) for r in reqs], [])
        rates, lat = [], []
        for _ in range(3):
            t0 = time.perf_counter()
            tickets = [submit(srv, r) for r in reqs]
            lat_pass = []
            drain(tickets, lat_pass)
            rates.append(len(reqs) / (time.perf_counter() - t0))
            lat += lat_pass
        srv.close()
        return statistics.median(rates), rates, lat

    reqs = [make_req() for _ in range(sat_requests)]
    sat_rate, rates, lat_sat = saturation(reqs)
    traces = {}

    def poisson(frac, plain_mode=False, base_rate=None, max_requests=None):
        """Poisson arrivals at frac x base_rate (default: the saturation rate) for `seconds`;
        submit->result latencies."""
        rate = frac * (base_rate or sat_rate)
        n_req = max(50, int(rate * seconds))
        if max_requests:
            n_req = min(n_req, max_requests)
        if plain_mode and base_rate is None and frac in traces:  # the product server's requests and arrival times
            reqs, arrivals = traces[frac]
            reqs, arrivals = reqs[:n_req], arrivals[:n_req]
        else:
            reqs = [make_req() for _ in range(n_req)]
            arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
            if not plain_mode:
                traces[frac] = (reqs, arrivals)
        srv = new_server(plain_mode)
        for r in reqs[:16]:
            submit(srv, r).wait(120000)
        lat = []
        queue = []
        queued = []  # submit -> admission into a tick, per request
        lock = threading.Condition()
        done_flag = [False]

        def waiter():
            while True:
                with lock:
                    while not queue and not done_flag[0]:
                        lock.wait()
                    if not queue and done_flag[0]:
                        return
                    t = queue.pop(0)
                t.wait(120000)
                lat.append(t.result.latency_ms)
                queued.append(t.result.queue_ms)

        th = threading.Thread(target=waiter)
        th.start()
        t0 = time.perf_counter()
        for r, at in zip(reqs, arrivals):
            while time.perf_counter() - t0 < at:
                pass
            tk = submit(srv, r)
            with lock:
                queue.append(tk)
                lock.notify()
        with lock:
            done_flag[0] = True
            lock.notify()
        th.join()
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lat = np.array(lat)
        return {"load": frac, "offered_rate_per_s": rate, "requests": int(n_req),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "achieved_drrs_per_s": n_req / wall, "ticks": int(st["ticks"]),
                "gpu_busy_frac": st["gpu_busy_ms"] / 1e3 / wall,
                "queue_p50_ms": float(np.percentile(queued, 50)), "queue_p99_ms": float(np.percentile(queued, 99)),
                "max_ms": float(lat.max())}

    runs = [poisson(f) for f in loads]
    head = next((r for r in runs if r["load"] == 0.5), runs[0])
    plain_res = None
    if plain:
        # the comparison server, measured through the same request loop: its own
        # saturation, Poisson load at half of it, and the product server's headline
        # request stream (which it cannot keep up with: latencies grow with the run)
        p_sat, p_rates, _ = saturation(reqs[:300], plain_mode=True)
        own = poisson(0.5, plain_mode=True, base_rate=p_sat)
        same = poisson(head["load"], plain_mode=True, max_requests=1000)
        plain_res = {"saturation_drrs_per_s": p_sat, "saturation_passes_per_s": p_rates,
                     "at_half_own_saturation": own, "at_product_headline_rate": same,
                     "what": "drr_server with plain_fp32_baseline: one request per tick, plain FP32 forward walk, "
                             "gradients by central differences (13 renders per pose); same request mix"}
    reg = registration_step_latency(drr, vols)
    lone = lone_request_latency(drr, vols)
    return {"p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"], "mean_ms": head["mean_ms"],
            "requests": head["requests"], "offered_rate_per_s": head["offered_rate_per_s"],
            "achieved_drrs_per_s": head["achieved_drrs_per_s"], "saturation_drrs_per_s": sat_rate,
            "saturation_p50_ms": float(np.percentile(lat_sat, 50)), "saturation_passes_per_s": rates,
            "ticks": head["ticks"],
            "gpu_busy_frac": head["gpu_busy_frac"], "by_load": runs, "plain_fp32_server": plain_res,
            "registration_step": reg, "lone_requests": lone,
            "max_tick_work": max_tick_work,
            "tick_depth": tick_depth or 3,
            "workload": "8 resident volumes {128^3, 256^3, 512x512x133, 512x512x300} x {FP32, BF16}; one pose per "
                        "request; detector H=W~U{128..512} at 280/H mm, SDR 510; 50% render+pose-grad; Poisson "
                        "arrivals at the listed fractions of the measured saturation rate (headline: 50%)"}


def lone_request_latency(drr, vols, sizes=(128, 256, 512), reps=20):
    """One request at a time on the 256^3 FP32 volume: the direct calls' device time
    (CUDA events around the call, pose setup included; the fwd+grad call takes the split
    walk where it applies) and the served submit->result latency, with the loop sleeping
    until woken (the default) and with spin_poll_us = 500."""
    import torch
    from paper_2208_12737_gb300 import inputs
    vol = dict(vols)["256^3/f32"]
    out = {}
    for n in sizes:
        det = inputs.Detector(510.0, n, n, 280.0 / n, 280.0 / n)
        P_np = inputs.random_poses(1, seed=5)
        P = torch.from_numpy(P_np).cuda()
        g = torch.from_numpy(inputs.upstream_grad((1, n, n), seed=n)).cuda()
        E = torch.empty((1, n, n), device="cuda")
        J = torch.empty((1, 6, n, n), device="cuda")

        def fwd():
            drr.render(vol, det, P, out=E)

        def fwdgrad():
            drr.render(vol, det, P, jacobian=True, out=E, jac=J)
            drr.render_backward(vol, det, P, g, jac=J)

        row = {}
        for name, fn in (("direct_render_ms", fwd), ("direct_render_pose_grad_ms", fwdgrad)):
            for _ in range(5):
                fn()
            ms = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn()
                b.record()
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            row[name] = statistics.median(ms)
        buf = np.zeros((1, n, n), np.float32)
        for name, spin in (("served_render_ms", 0), ("served_render_spin_poll_ms", 500)):
            srv = drr.Server(device_budget=256 << 20, spin_poll_us=spin)
            lat = []
            for i in range(reps + 5):
                t = srv.submit(vol, det, P_np, out=buf)
                t.wait(60000)
                if i >= 5:
                    lat.append(t.result.latency_ms)
            srv.close()
            row[name] = statistics.median(lat)
        out[f"{n}x{n}"] = row
    out["workload"] = "256^3 ellipsoid phantom (FP32, 1 mm), one pose per request, n x n detector at 280/n mm, SDR 510"
    return out


def run_lone_only():
    """The lone-request latencies on their own (only the 256^3 volume resident)."""
    from paper_2208_12737_gb300 import build, inputs
    build.build()
    from paper_2208_12737_gb300 import drr
    v = inputs.ellipsoid_phantom((256, 256, 256), (1.0, 1.0, 1.0), seed=82, semi_range=(10, 60),
                                 density_range=(0.0, 0.01))
    return {"lone_requests": lone_request_latency(drr, [("256^3/f32", drr.Volume(v, (1.0, 1.0, 1.0)))])}


def registration_step_latency(drr, vols, n=256, reps=20):
    """A lone registration-step request (fixed image in; E, -ZNCC and its pose gradient out)
    on the 512x512x133 FP32 volume at n x n, served one at a time: median submit->result
    latency, beside the same step as direct calls from host data (median wall time, synchronised)."""
    import torch
    from paper_2208_12737_gb300 import inputs
    vol = dict(vols)["512x512x133/f32"]
    det = inputs.Detector(510.0, n, n, 280.0 / n, 280.0 / n)
    truth = inputs.random_poses(1, seed=77)
    fixed = drr.render(vol, det, torch.from_numpy(truth).cuda()).cpu().numpy()
    moving = (truth + inputs.pose_offsets(1, seed=78, max_angle_deg=5, max_trans_mm=5)).astype(np.float32)
    srv = drr.Server(device_budget=1 << 30)
    lat = []
    for i in range(reps + 3):
        t = srv.submit(vol, det, moving, fixed=fixed)
        t.wait(60000)
        if i >= 3:
            lat.append(t.result.latency_ms)
    srv.close()
    fixed_d = torch.from_numpy(fixed).cuda()
    direct = []
    for i in range(reps + 3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        poses = torch.from_numpy(moving).cuda()
        E, J = drr.render(vol, det, poses, jacobian=True)
        loss, g = drr.zncc(E, fixed_d)
        G = drr.render_backward(vol, det, poses, g, jac=J)
        E.cpu(), G.cpu(), loss.cpu()
        if i >= 3:
            direct.append((time.perf_counter() - t0) * 1e3)
    return {"served_p50_ms": statistics.median(lat), "direct_calls_ms": statistics.median(direct),
            "workload": f"512x512x133 CT (FP32), {n}x{n} @ {280.0 / n:.3g} mm, one pose, -ZNCC against a "
                        "rendered fixed image (fixed image resident on the device for the direct calls)"}


def l2_read_gbs(drr, mb=64, reps=20):
    """Measured L2 read bandwidth (GB/s): a buffer that fits in L2, streamed reps times."""
    import torch
    buf = torch.zeros(mb << 20, dtype=torch.uint8, device="cuda")
    sink = torch.zeros(1, device="cuda")
    drr.probe_l2_read(buf, 2, sink)  # warm: brings the buffer into L2
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        drr.probe_l2_read(buf, reps, sink)
        b.record()
        torch.cuda.synchronize()
        best = max(best, reps * buf.numel() / (a.elapsed_time(b) * 1e-3) / 1e9)
    return best


def vgs_torch_forward(mu, spacing, det, poses, chunk=4):
    """The paper's vectorised Siddon (Sec. 2.3) written as plain PyTorch tensor ops on the GPU,
    as bench context only: every plane crossing of every ray (Eq. 3) is materialised, clamped to
    [alpha_min, alpha_max], sorted per ray, and Eq. 2 is evaluated on the midpoints.  FP32, like
    the paper's implementation.  mu: (nz, ny, nx) float32 tensor on the GPU; poses: (B, 6) tensor."""
    import torch
    dev = mu.device
    nz, ny, nx = mu.shape
    n = torch.tensor([nx, ny, nz], device=dev, dtype=torch.float32)
    delta = torch.tensor(spacing, device=dev, dtype=torch.float32)
    b0 = -0.5 * n * delta
    rho = 0.5 * det.sdr
    hh = (torch.arange(det.height, device=dev, dtype=torch.float32) - 0.5 * (det.height - 1)) * det.delta_h
    ww = (torch.arange(det.width, device=dev, dtype=torch.float32) - 0.5 * (det.width - 1)) * det.delta_w
    pc = torch.stack(torch.broadcast_tensors(torch.full((det.height, det.width), -rho, device=dev),
                                             ww[None, :].expand(det.height, -1), hh[:, None].expand(-1, det.width)),
                     dim=-1)  # (H, W, 3)
    planes = [b0[a] + torch.arange(int(n[a]) + 1, device=dev, dtype=torch.float32) * delta[a] for a in range(3)]
    flat = mu.reshape(-1)
    out = []
    for c0 in range(0, poses.shape[0], chunk):
        P = poses[c0:c0 + chunk].float()
        cz, sz = torch.cos(P[:, 0]), torch.sin(P[:, 0])
        cy, sy = torch.cos(P[:, 1]), torch.sin(P[:, 1])
        cx, sx = torch.cos(P[:, 2]), torch.sin(P[:, 2])
        o, z = torch.ones_like(cz), torch.zeros_like(cz)
        Rz = torch.stack([cz, -sz, z, sz, cz, z, z, z, o], -1).view(-1, 3, 3)
        Ry = torch.stack([cy, z, sy, z, o, z, -sy, z, cy], -1).view(-1, 3, 3)
        Rx = torch.stack([o, z, z, z, cx, -sx, z, sx, cx], -1).view(-1, 3, 3)
        R = Rz @ Ry @ Rx
        t = P[:, 3:]
        s = R[:, :, 0] * rho + t                                         # (b, 3)
        p = torch.einsum("bij,hwj->bhwi", R, pc) + t[:, None, None, :]  # (b, H, W, 3)
        d = p - s[:, None, None, :]
        sa = s[:, None, None, :].expand_as(d)
        with torch.no_grad():
            al = []
            lo = torch.zeros(d.shape[:-1], device=dev)
            hi = torch.ones(d.shape[:-1], device=dev)
            for a in range(3):
                A = (planes[a][None, None, None, :] - sa[..., a:a + 1]) / d[..., a:a + 1]
                al.append(A)
                lo = torch.maximum(lo, torch.minimum(A[..., 0], A[..., -1]))
                hi = torch.minimum(hi, torch.maximum(A[..., 0], A[..., -1]))
            A = torch.cat(al + [lo[..., None], hi[..., None]], dim=-1)
            A = torch.minimum(torch.maximum(A, lo[..., None]), hi[..., None])
            A, _ = torch.sort(A, dim=-1)
            mid = 0.5 * (A[..., 1:] + A[..., :-1])
            x = sa[..., None, :] + mid[..., None] * d[..., None, :]
            idx = torch.floor((x - b0) / delta).long()
            inside = ((idx >= 0) & (idx < n.long())).all(dim=-1)
            lin = (idx[..., 2] * ny + idx[..., 1]) * nx + idx[..., 0]
            v = torch.where(inside, flat[lin.clamp(0, flat.numel() - 1)], torch.zeros((), device=dev))
            E = (v * (A[..., 1:] - A[..., :-1])).sum(-1) * d.norm(dim=-1)
        out.append(E)
    return torch.cat(out)


def vgs_baseline(drr, hu, cfg, poses, E_ours, rays, reps=2):
    """Times the vectorised-tensor Siddon above on the same batch; reports its agreement with
    the kernel's DRR (max relative difference with the 1e-3 * max floor)."""
    import torch
    from paper_2208_12737_gb300 import inputs
    mu = torch.from_numpy(np.maximum(0.0, inputs.MU_WATER * (1.0 + hu.astype(np.float32) / 1000.0))
                          .astype(np.float32)).cuda()
    det = cfg["detector"]
    E = vgs_torch_forward(mu, cfg["spacing"], det, poses)  # warm-up
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        E = vgs_torch_forward(mu, cfg["spacing"], det, poses)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    ref = E_ours.double()
    floor = 1e-3 * ref.abs().max()
    diff = float(((E.double() - ref).abs() / torch.maximum(ref.abs(), floor)).max())
    del mu, E
    torch.cuda.empty_cache()
    return {"ms_per_step": t, "value": rays / (t * 1e-3) / 1e9, "unit": UNIT, "max_rel_diff_vs_kernel": diff,
            "what": "forward only: the paper's vectorised Siddon as plain PyTorch ops (FP32, materialise, "
                    "clamp, sort, Eq. 2 on midpoints), 4 poses per pass"}


def plain_fp32_baseline(drr, vol, det, poses, E_ours, rays, reps=5):
    """The plain FP32 forward walk on the same batch (the comparison baseline), with its
    largest relative difference from the product kernel's DRR (1e-3 * max floor)."""
    import torch
    out = torch.empty_like(E_ours)
    drr.render_plain_fp32(vol, det, poses, out=out)
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        drr.render_plain_fp32(vol, det, poses, out=out)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    ref = E_ours.double()
    floor = 1e-3 * ref.abs().max()
    diff = float(((out.double() - ref).abs() / torch.maximum(ref.abs(), floor)).max())
    return {"ms_per_step": t, "value": rays / (t * 1e-3) / 1e9, "unit": UNIT, "max_rel_diff_vs_kernel": diff,
            "what": "forward only: textbook incremental Siddon-Jacobs walk, all FP32, thread per ray, linear layout"}


def precision_bench(drr, reps=3):
    """The precision-sweep workload (512^3 at 0.5 mm, 1024x1024 at 0.4 mm, 8 poses): forward
    throughput per storage dtype and the largest relative difference from the FP32-storage DRR
    (the errors against the FP64 oracle are the parity tests' business)."""
    import torch
    from paper_2208_12737_gb300 import inputs
    cfg = inputs.PRECISION
    vol_np = inputs.bone_tissue_phantom(cfg["shape_zyx"], cfg["spacing"], seed=cfg["phantom_seed"])
    det = cfg["detector"]
    poses = torch.from_numpy(inputs.random_poses(cfg["batch"], seed=cfg["pose_seed"])).cuda()
    rays = cfg["batch"] * det.height * det.width
    res = {}
    E32 = None
    for storage in ("f32", "bf16", "f16"):
        v = drr.Volume(vol_np, cfg["spacing"], storage=storage)
        E = drr.render(v, det, poses)
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            drr.render(v, det, poses, out=E)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        t = statistics.median(ms)
        if E32 is None:
            E32 = E.double()
        floor = 1e-3 * E32.abs().max()
        res[storage] = {"fwd_ms": t, "grays_per_s": rays / (t * 1e-3) / 1e9,
                        "max_rel_diff_vs_f32": float(((E.double() - E32).abs() / torch.maximum(E32.abs(), floor)).max())}
        v.close()
    res["workload"] = "512^3 at 0.5 mm (air / soft tissue 0.02 / bone 0.04-0.06 per mm), 1024x1024 at 0.4 mm, 8 poses"
    return res


def adjoint_bench(drr, vol, det, poses, g, hu_shape, rays, reps=3):
    """The volume adjoint (back-projection into a zeroed FP32 gradient volume, one atomic add
    per segment) on the headline batch."""
    import torch
    gv = torch.zeros(hu_shape, device=poses.device, dtype=torch.float32)
    drr.render_backward(vol, det, poses, g, pose_grad=False, grad_volume=gv)
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        gv.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        drr.render_backward(vol, det, poses, g, pose_grad=False, grad_volume=gv)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    return {"ms_per_step": t, "value": rays / (t * 1e-3) / 1e9, "unit": UNIT,
            "what": "dL/dV by back-projection (FP32 chunked re-walk, FP32 atomics merged down 4x8-tile pixel columns) for the 16-pose batch"}


def fd_baseline(drr, vol, det, poses, rays, reps=3, plain=False):
    """The finite-difference alternative to the analytic pose gradient: central differences
    need 12 extra forward renders per pose (13 with the DRR itself), timed as one batch;
    with plain=True on the plain FP32 forward walk instead of the exact one."""
    import torch
    P = poses.repeat(13, 1).contiguous()
    steps = torch.tensor([1e-3] * 3 + [1e-2] * 3, device=poses.device)
    for k in range(6):
        P[(1 + 2 * k) * len(poses):(2 + 2 * k) * len(poses), k] += steps[k]
        P[(2 + 2 * k) * len(poses):(3 + 2 * k) * len(poses), k] -= steps[k]
    out = torch.empty((P.shape[0], det.height, det.width), device=poses.device)
    render = drr.render_plain_fp32 if plain else drr.render
    render(vol, det, P, out=out)
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        render(vol, det, P, out=out)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    walk = "the plain FP32 forward walk" if plain else "the exact forward walk"
    return {"ms_per_step": t, "value": rays / (t * 1e-3) / 1e9, "unit": UNIT,
            "what": f"DRR + central-difference pose gradient: 13 renders per pose by {walk} "
                    "(h = 1e-3 rad, 1e-2 mm)"}


def registration_bench(drr, hu, lr_rot=1e-2, lr_trans=1.0):
    """The registration workload: 64 concurrent registrations on the CT volume, 256x256
    detector, initial offsets U(+-15 deg, +-20 mm) from seeded ground truths, -ZNCC with
    Adam for 200 steps; convergence is -ZNCC < -0.999."""
    import torch
    from paper_2208_12737_gb300 import inputs
    cfg = inputs.REGISTRATION
    vol = drr.Volume(hu, cfg["spacing"], hu=True)
    det = cfg["detector"]
    B, steps = cfg["batch"], cfg["steps"]
    truth = inputs.random_poses(B, seed=cfg["truth_seed"])
    init = truth + inputs.pose_offsets(B, seed=cfg["offset_seed"])
    fixed = drr.render(vol, det, torch.from_numpy(truth).cuda())
    drr.register(vol, det, fixed, torch.from_numpy(init).cuda(), steps=3)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    poses, hist, first = drr.register(vol, det, fixed, torch.from_numpy(init).cuda(), steps=steps,
                                      lr_rot=lr_rot, lr_trans=lr_trans)
    dt = time.perf_counter() - t0
    conv = first >= 0
    err = poses - truth
    return {"registrations": B, "steps": steps, "steps_per_s": steps / dt, "registration_steps_per_s": B * steps / dt,
            "converged": int(conv.sum()), "mean_steps_to_converge": float(first[conv].mean()) if conv.any() else None,
            "final_loss_median": float(np.median(hist[-1])),
            "rot_err_deg_median": float(np.rad2deg(np.median(np.abs(err[:, :3])))),
            "trans_err_mm_median": float(np.median(np.abs(err[:, 3:]))),
            "optimizer": f"Adam lr_rot={lr_rot} rad, lr_trans={lr_trans} mm, betas (0.9, 0.999)",
            "workload": "512x512x133 CT, 256x256 @1.4 mm, SDR 510; 64 problems, offsets U(+-15 deg, +-20 mm)"}


def landscape_bench(drr, hu, reps=3):
    """The loss-landscape workload (Sec. 3.2): -ZNCC of 4096 DRRs (200x200) of the CT at
    displacements U(90, 90, 45 deg; 30 mm widths) around one pose against the DRR at that pose."""
    import torch
    from paper_2208_12737_gb300 import inputs
    cfg = inputs.LANDSCAPE
    vol = drr.Volume(hu, cfg["spacing"], hu=True)
    det = cfg["detector"]
    truth = inputs.random_poses(1, seed=cfg["truth_seed"])
    poses = torch.from_numpy((truth + inputs.landscape_offsets(cfg["n"], seed=cfg["offset_seed"])).astype(np.float32))
    poses = poses.cuda()
    fixed = drr.render(vol, det, torch.from_numpy(truth).cuda())[0]
    out = torch.empty((cfg["n"],), device="cuda")
    drr.loss_landscape(vol, det, fixed, poses, out=out)  # warm-up
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        drr.loss_landscape(vol, det, fixed, poses, out=out)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    L = out.cpu().numpy()
    rays = cfg["n"] * det.height * det.width
    return {"poses": cfg["n"], "ms": t, "drrs_per_s": cfg["n"] / (t * 1e-3), "grays_per_s": rays / (t * 1e-3) / 1e9,
            "loss_min": float(L.min()), "loss_median": float(np.median(L)),
            "workload": "512x512x133 CT, 200x200 @1.4 mm, SDR 510; 4096 displacements U(90,90,45 deg; 30 mm)"}


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2208_12737_gb300 import build
    build.build()
    from paper_2208_12737_gb300 import drr

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    cfg, hu, poses_np, g_np = workload_inputs(rank)
    det = cfg["detector"]
    B, H, W = cfg["batch"], det.height, det.width
    rays = B * H * W
    vol = drr.Volume(hu, cfg["spacing"], hu=True, storage=args.storage)
    poses = torch.from_numpy(poses_np).to(dev)
    g = torch.from_numpy(g_np).to(dev)
    E = torch.empty((B, H, W), device=dev)
    J = torch.empty((B, 6, H, W), device=dev)

    def step():
        drr.render(vol, det, poses, jacobian=True, out=E, jac=J)
        return drr.render_backward(vol, det, poses, g, jac=J)

    def fwd():
        drr.render(vol, det, poses, out=E)

    # inputs larger than L2 are not the case here (the volume is meant to stay L2-resident
    # between renders); L2 is flushed before every timed step instead, outside the events.
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    seg = drr.count_segments(vol, det, poses).to(torch.int64).sum().item()  # outside the timed region
    elem = {"f32": 4, "bf16": 2, "f16": 2}[args.storage]

    for _ in range(args.warmup):
        step()
        fwd()
    torch.cuda.synchronize()

    def timed(fn, k):
        return timed_steps(fn, k, before=lambda i: flush.fill_(float(i)))

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    launches0 = drr.launch_count()
    t0 = time.perf_counter()
    step_ms = timed(step, args.steps)
    wall = time.perf_counter() - t0
    launches = drr.launch_count() - launches0
    # the same K steps again with CUDA events around every launch (on the launch
    # stream) for the per-kernel durations; those events add ~15 us to a step, so
    # the headline steps above run without them
    drr.profile_reset()
    drr.profile_enable(True)
    timed(step, args.steps)
    drr.profile_enable(False)
    kern_ms, kern_n = drr.profile_read("siddon_fwd_jac")
    red_ms, red_n = drr.profile_read("jac_reduce")
    ps_ms, ps_n = drr.profile_read("pose_setup")
    fwd_ms = timed(fwd, args.steps)
    # end-to-end through the public API: pinned host poses in, DRR + pose gradient out
    poses_h = torch.from_numpy(poses_np).pin_memory()
    E_h = torch.empty((B, H, W), dtype=torch.float32).pin_memory()
    G_h = torch.empty((B, 6), dtype=torch.float32).pin_memory()
    poses_d = torch.empty_like(poses)

    copy_stream = torch.cuda.Stream()
    e_ready = torch.cuda.Event()

    def e2e():
        # the poses are read from, and E and dL/d eta written to, pinned host memory by the
        # kernels themselves (across NVLink-C2C): no staging copies
        drr.render(vol, det, poses_h, jacobian=True, out=E_h, jac=J)
        drr.render_backward(vol, det, poses_h, g, jac=J, grad_pose_out=G_h)

    def e2e_staged():
        # the same with staging copies: poses up, then the DRR back on a side stream while
        # the gradient reduction runs, then dL/d eta back
        main = torch.cuda.current_stream()
        poses_d.copy_(poses_h, non_blocking=True)
        drr.render(vol, det, poses_d, jacobian=True, out=E, jac=J)
        e_ready.record(main)
        copy_stream.wait_event(e_ready)
        with torch.cuda.stream(copy_stream):
            E_h.copy_(E, non_blocking=True)
        G = drr.render_backward(vol, det, poses_d, g, jac=J)
        G_h.copy_(G, non_blocking=True)
        main.wait_stream(copy_stream)

    for _ in range(args.warmup):
        e2e()
        e2e_staged()
    torch.cuda.synchronize()
    e2e_ms = timed(e2e, args.steps)
    e2e_staged_ms = timed(e2e_staged, args.steps)
    # the same step captured once in a CUDA graph and replayed (no host launch work per step)
    graph_ms = None
    try:
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            step()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        graph_ms = statistics.mean(timed(graph.replay, args.steps))
    except RuntimeError as exc:  # capture refused: report the reason instead of a number
        graph_ms = str(exc).splitlines()[0]
    torch.cuda.synchronize()
    clk = clocks.stop()
    drr.profile_reset()

    (ms, fms, ems, sms), (value, fwd_value, e2e_value, staged_value) = job_timing(
        world, rays, [step_ms, fwd_ms, e2e_ms, e2e_staged_ms], dist, dev)
    # the gather roofline's L2 ceiling, measured in the same run
    l2 = l2_read_gbs(drr)
    if dist:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return
    peaks, which = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # dominant kernel: the fused forward + Jacobian walk.  Its algorithmic bytes per
    # launch are the voxel gathers of Eq. 2, one storage element per segment.
    k_ms = kern_ms / max(kern_n, 1)
    gather_gbs = seg * elem / (k_ms * 1e-3) / 1e9
    ops_per_seg = 8  # 3-way min (2), length (1), accumulate (1), next crossing (1), Jacobian weight and sums (3)
    peak_alu = 152 * 128 * sm_max * 1e6 / 1e12  # FP32 lanes x max SM clock, tera-ops/s
    vol_bytes = int(np.prod(hu.shape)) * elem
    issue = issue_roofline(k_ms, sm_max)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.storage == "f32" else f"{args.storage}-storage/f32-accum",
        "data": "synthetic",
        "config": {"workload": cfg["name"], "volume": "512x512x133 int16 HU -> FP32 /mm, 0.703x0.703x2.5 mm",
                   "detector": "200x200 @ 1.4 mm, SDR 510 mm", "batch": B, "rays_per_step": rays,
                   "segments_per_step": int(seg), "storage": args.storage,
                   "step": "pose setup + fused Siddon fwd with per-ray pose Jacobian + g.J reduction",
                   "l2": "flushed (512 MB write) before every timed step, outside the timed events"},
        "fwd_only": {"value": fwd_value, "unit": UNIT, "ms_per_step": fms},
        "drrs_per_s": world * B / (ms * 1e-3),
        "segments_per_s": world * seg / (ms * 1e-3),
        # Gather roofline: voxel bytes gathered per second by the dominant kernel (segments x
        # element size / its event-timed launch) against the measured HBM copy bandwidth, and
        # beside it against the L2 read bandwidth probed in this run.  What binds the kernel is
        # instruction issue (`issue`: ncu warp instructions per launch / launch time / the issue
        # peak of 4 schedulers x SMs x max clock); the gathers stay well below both ceilings.
        "roofline": {"bound": "hbm", "achieved": gather_gbs, "peak": hbm, "unit": "GB/s",
                     "frac": gather_gbs / hbm, "traffic": profiled_traffic("siddon_fwd_jac"),
                     "kernel": "siddon_fwd_jac", "kernel_ms": k_ms,
                     "algorithmic_bytes_per_launch": int(seg) * elem,
                     "unit_of_work": f"{int(seg)} segments x {elem} B voxel gather",
                     "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({which})",
                     "l2": {"achieved_gbs": gather_gbs, "peak_gbs": l2, "frac": gather_gbs / l2,
                            "peak_source": "measured in this run: 64 MB L2-resident buffer streamed with "
                                           "16-byte L2-only loads (drr_probe_l2_read)"},
                     "limiter": "issue",
                     "issue": issue,
                     # aside: a hand-counted 8 essential FP32 ops per segment against the FP32 lanes
                     "alu_aside": {"ops_per_segment": ops_per_seg,
                                   "achieved_tops": seg * ops_per_seg / (k_ms * 1e-3) / 1e12,
                                   "peak_tops": peak_alu,
                                   "frac": seg * ops_per_seg / (k_ms * 1e-3) / 1e12 / peak_alu},
                     # the volume's compulsory first touch from HBM after the flush, per kernel launch
                     "compulsory_hbm": {"bytes": vol_bytes, "achieved_gbs": vol_bytes / (k_ms * 1e-3) / 1e9,
                                        "peak_gbs": hbm, "frac": vol_bytes / (k_ms * 1e-3) / 1e9 / hbm}},
        "step_ms_stats": {"mean": statistics.mean(step_ms), "median": statistics.median(step_ms),
                          "p99": float(np.quantile(step_ms, 0.99)), "min": min(step_ms), "max": max(step_ms),
                          "rank": rank},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": B * 6 * 4,
                "d2h_bytes_per_step": B * H * W * 4 + B * 6 * 4,
                "how": "drr.render / drr.render_backward on pinned host poses, E and dL/d eta: the kernels read "
                       "and write them in place across the host link (the J planes stay on the device)",
                "staged_copies": {"value": staged_value, "unit": UNIT, "how": "device buffers, cudaMemcpyAsync of the poses up and of "
                                                       "E (side stream) and dL/d eta down"}},
        "graph_replay": ({"ms_per_step": graph_ms, "value": job_throughput(1, rays, graph_ms), "unit": UNIT}
                         if isinstance(graph_ms, float) else {"unavailable": graph_ms}),
        "step_kernels_ms": {"pose_setup": ps_ms / max(ps_n, 1), "siddon_fwd_jac": kern_ms / max(kern_n, 1),
                            "jac_reduce": red_ms / max(red_n, 1)},
        # the paper's own timing, other hardware and another CT: context, not a baseline
        "paper_context": {"what": "vectorised PyTorch Siddon forward, 200x200 DRR of a chest CT (Table 1)",
                          "ms": 72.7, "grays_per_s": 200 * 200 / 72.7e-3 / 1e9, "hardware": "RTX 2080 Ti",
                          "pose_gradient_autograd_ms": 35.1, "pose_gradient_size": "unstated"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "wall_s_timed": wall,
    }
    if not args.no_baselines:
        line["fd_baseline"] = fd_baseline(drr, vol, det, poses, rays)
        line["fd_baseline_plain_fp32"] = fd_baseline(drr, vol, det, poses, rays, plain=True)
        line["volume_adjoint"] = adjoint_bench(drr, vol, det, poses, g, hu.shape, rays)
        drr.render(vol, det, poses, out=E)
        line["plain_fp32_baseline"] = plain_fp32_baseline(drr, vol, det, poses, E, rays)
        if not args.no_vgs:
            drr.render(vol, det, poses, out=E)
            line["vgs_torch_baseline"] = vgs_baseline(drr, hu, cfg, poses, E, rays)
    if not args.no_precision:
        line["precision"] = precision_bench(drr)
    if not args.no_registration:
        line["registration"] = registration_bench(drr, hu)
    if not args.no_landscape:
        line["landscape"] = landscape_bench(drr, hu)
    if not args.no_serve:
        line["served"] = serve_bench(drr, hu, seconds=args.serve_seconds)
        line["served_p50_ms"] = line["served"]["p50_ms"]
        line["served_p99_ms"] = line["served"]["p99_ms"]
    if not args.no_cpu_baseline:
        cb, _, _ = cpu_oracle_sample(cfg, hu, poses_np, seconds_target=args.cpu_seconds)
        line["cpu_baseline"] = cb
        cb1, _, _ = cpu_oracle_sample(cfg, hu, poses_np, seconds_target=args.cpu_seconds / 2, threads=1)
        line["cpu_baseline_1core"] = cb1
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", choices=["f32", "bf16", "f16"], default="f32")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-registration", action="store_true")
    ap.add_argument("--no-landscape", action="store_true")
    ap.add_argument("--no-vgs", action="store_true", help="skip the vectorised-tensor Siddon context line")
    ap.add_argument("--no-baselines", action="store_true",
                    help="skip the FD, plain-FP32, volume-adjoint and vectorised baselines (the L2 probe always runs)")
    ap.add_argument("--no-precision", action="store_true", help="skip the 512^3 precision-sweep workload")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="seconds per served load level")
    ap.add_argument("--lone-only", action="store_true",
                    help="only the lone-request latencies (one JSON object; a small case for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.lone_only:
        print(json.dumps(run_lone_only()), flush=True)
        return
    rank, world, local_rank = resolve_world(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
