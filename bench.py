"""Benchmark of the MPPI step on GB300.

Headline workload (one "step" = one control step of a closed loop): the
figure-eight tracking problem with 64 spherical obstacles, K=16384 samples,
N=100, dt=0.01 s, per-motor thrust limits.  Each step solves one MPPI
iteration on device-resident inputs (state, reference window, obstacles,
warm-start nominal), then the simulated vehicle advances by the applied
command (the kernel's x_next) and the warm start is the shifted nominal.

Printed: one JSON line with rollout-steps/s (K*N per second), solves/s,
p50/p99 latency, an end-to-end figure through the host-buffer C ABI, the
roofline of the fused kernel, the CPU oracle timed on the host cores, the
batched (256 uneven instances, persistent kernel, CUDA graph) and served
(continuous batching) forms, and the SM clocks seen during the timed region.

`--impl reference` times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MPPI rollout-steps/s, solves/s, p50/p99 solve latency: batched vs plain, 1 GB300"
UNIT = "rollout-steps/s"
K_HEAD, N_HEAD, DT_HEAD, M_HEAD = 16384, 100, 0.01, 64
WORKLOAD = ("closed-loop figure-eight tracking, K=16384, N=100, dt=0.01 s, 64 spheres, "
            "per-motor thrust limits, lambda=1")

# Algorithmic FP32 work per rollout-step and per evaluated (state,
# obstacle) pair, counted from the equations of the method as the oracle
# writes them: per rollout step noise 24, perturb + clamp 12, input and rate
# cost 27, constraint pipeline 95, RK4 437, renormalisation 12, tracking
# cost 43; per pair 17.  Pairs whose barrier term is below its floor (2^-48
# of c_bar, where it counts as zero) and that cannot be in collision are not
# part of the result and are not counted; the kernel reports how many pairs
# it evaluated (mppi_set_counters).
FLOP_PER_STEP = 650
FLOP_PER_PAIR = 17
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the headline kernel in an ncu capture of this workload: the inputs, the
# partials and the outputs; everything else stays on chip.  Taken for the
# kernel as it is; set to None when the kernel changes until recaptured.
HEADLINE_TRAFFIC_BYTES = 122624
SMS, LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0


def fp32_peak_tflops(mhz: float = SM_MAX_MHZ) -> float:
    return SMS * LANES_PER_SM * 2 * mhz * 1e6 / 1e12


# ---------------------------------------------------------------- helpers

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0:  # first sample before timing starts
                time.sleep(0.005)
            self.lines.clear()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier_max(value: float, world: int) -> float:
    """Largest value over the ranks (the slowest rank's time)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.barrier()
        if torch.cuda.is_available():
            torch.cuda.synchronize()


def whole_job_rate(units_per_step_per_rank: float, steps: int, max_ms: float, world: int) -> float:
    """Units processed by all ranks divided by the slowest rank's time
    (replicas: every rank solves its own vehicle; weak scaling)."""
    return world * units_per_step_per_rank * steps / (max_ms * 1e-3)


# --------------------------------------------------------------- workload

def headline_problem(rank: int):
    from paper_2407_09812_gb300 import inputs as I
    prob = I.eight_with_spheres(K=K_HEAD, N=N_HEAD, dt=DT_HEAD, M=M_HEAD, seed=1, stream_id=rank)
    return prob


def reference_windows(n_steps: int):
    from paper_2407_09812_gb300 import inputs as I
    traj = I.Trajectory("eight")
    return np.stack([traj.window(DT_HEAD * t, N_HEAD, DT_HEAD) for t in range(n_steps)])


def run_closed_loop(args, rank):
    import torch
    from paper_2407_09812_gb300 import mppi

    dev = torch.device("cuda")
    prob = headline_problem(rank)
    n_total = args.warmup + args.steps
    refs = torch.from_numpy(reference_windows(n_total)).to(dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    obs = t(prob["obstacles"])
    x = [t(prob["x_hat"]), torch.zeros(13, device=dev)]
    u = [t(prob["u_nom"]), torch.zeros(N_HEAD, 4, device=dev)]
    u_out = torch.zeros(N_HEAD, 4, device=dev)
    u_cmd = torch.zeros(4, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    solver = mppi.Solver(prob["model"], prob["params"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_total)]

    def step(i):
        a, b = i % 2, (i + 1) % 2
        solver.solve_async(x[a], refs[i], obs, u[a], i, u_out=u_out, u_cmd=u_cmd, u_next=u[b], x_next=x[b],
                           status=status, stream=stream)

    pairs = torch.zeros(1, dtype=torch.int64, device=dev)
    solver.set_counters(pairs)  # evaluated obstacle pairs, counted in the warm-up only
    for i in range(args.warmup):
        flush.zero_()
        step(i)
    torch.cuda.synchronize()
    pairs_per_solve = int(pairs.item()) / args.warmup
    solver.set_counters(None)
    barrier(args.world)
    with ClockSampler(torch.cuda.current_device()) as clk:
        wall0 = time.perf_counter()
        for i in range(args.warmup, n_total):
            flush.zero_()  # L2 flush between timed steps, outside the events
            ev[i][0].record(stream)
            step(i)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    barrier(args.world)
    ms = np.array([ev[i][0].elapsed_time(ev[i][1]) for i in range(args.warmup, n_total)])
    st = int(status.item())
    final_x = x[n_total % 2].cpu().numpy()
    solver.close()
    return {"ms": ms, "wall": wall, "clocks": clk.summary(), "status": st, "final_x": final_x,
            "x_trace_ok": bool(np.all(np.isfinite(final_x))), "pairs_per_solve": pairs_per_solve}


def run_e2e(args, rank, n_steps):
    """Same closed loop through mppi_solve with HOST buffers: every step
    copies its inputs host->device and its results device->host."""
    from paper_2407_09812_gb300 import mppi
    prob = headline_problem(rank)
    refs = reference_windows(n_steps + 3)
    solver = mppi.Solver(prob["model"], prob["params"])
    x, u = prob["x_hat"].copy(), prob["u_nom"].copy()
    lat = []
    for i in range(n_steps + 3):
        t0 = time.perf_counter()
        out = solver.solve(x, refs[i], prob["obstacles"], u, i)
        dt = time.perf_counter() - t0
        x, u = out["x_next"], out["u_next"]
        if i >= 3:
            lat.append(dt)
    solver.close()
    # Bytes of the two copies mppi_solve makes (16-byte aligned segments):
    # in: x_hat and the Philox counter, reference, obstacles, nominal; out:
    # u_out, u_cmd, u_next, x_next, status.
    N, M = N_HEAD, M_HEAD
    up4 = lambda v: (v + 3) // 4 * 4
    h2d = 4 * up4(up4(up4(16 + 13 * (N + 1)) + 4 * M) + 4 * N)
    d2h = 4 * (up4(4 * N) + 4 + up4(4 * N) + 16 + 4)
    lat = np.array(lat)
    return {"value": K_HEAD * N_HEAD / float(lat.mean()), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": float(lat.mean() * 1e3),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "api": "mppi_solve (host buffers, synchronous)"}


def run_batched(args, reps=5):
    """256 uneven instances (K log-uniform 1024..32768, N 30..150, 0..128
    spheres) in one persistent launch replayed from a CUDA graph, against
    solving the same instances one launch each."""
    import torch
    from paper_2407_09812_gb300 import inputs as I
    from paper_2407_09812_gb300 import mppi
    dev = torch.device("cuda")
    probs = I.batched_uneven(n=256, seed=2)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    insts = []
    for p in probs:
        N = p["params"]["N"]
        insts.append({"x_hat": t(p["x_hat"]), "ref": t(p["ref"]), "u_nom": t(p["u_nom"]),
                      "obstacles": t(p["obstacles"]) if p["obstacles"].size else None,
                      "u_out": torch.zeros(N, 4, device=dev), "u_cmd": torch.zeros(4, device=dev),
                      "K": p["params"]["K"], "N": N, "dt": p["params"]["dt"], "lambda": p["params"]["lambda"],
                      "sigma": p["params"]["sigma"], "seed": p["params"]["seed"],
                      "stream_id": p["params"]["stream_id"], "iter": p["iter"]})
    sumK = sum(i["K"] for i in insts)
    steps = sum(i["K"] * i["N"] for i in insts)
    cap = {"max_instances": len(insts), "max_samples": sumK, "N_max": 150, "M_max": 128}
    m = probs[0]["model"]
    solver = mppi.Solver(m, probs[0]["params"], cap)
    stream = torch.cuda.current_stream()
    pairs = torch.zeros(1, dtype=torch.int64, device=dev)
    solver.set_counters(pairs)
    solver.solve_batch(insts, stream=stream, graph=False)
    torch.cuda.synchronize()
    pairs_per_launch = int(pairs.item())
    solver.set_counters(None)
    for _ in range(2):
        solver.solve_batch(insts, stream=stream, graph=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        solver.solve_batch(insts, stream=stream, graph=True)
    e1.record()
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1) / reps
    # Plain: the same instances, one single-instance launch each.
    plain = mppi.Solver(m, probs[0]["params"], {"max_instances": 1, "max_samples": 32768, "N_max": 150,
                                                "M_max": 128})

    def plain_pass():
        for p, i in zip(probs, insts):
            plain.set_params(p["params"])
            plain.solve_async(i["x_hat"], i["ref"], i["obstacles"], i["u_nom"], i["iter"], u_out=i["u_out"],
                              u_cmd=i["u_cmd"], stream=stream)

    plain_pass()
    torch.cuda.synchronize()
    e0.record()
    plain_pass()
    e1.record()
    torch.cuda.synchronize()
    ms_p = e0.elapsed_time(e1)
    plain.close()
    solver.close()
    all_pairs = sum(i["K"] * (i["N"] + 1) * (0 if i["obstacles"] is None else i["obstacles"].shape[0])
                    for i in insts)
    flop = steps * FLOP_PER_STEP + pairs_per_launch * FLOP_PER_PAIR
    return {"workload": "256 uneven instances, K log-uniform [1024, 32768], N U[30,150], dt=0.01, 0-128 spheres",
            "instances": len(insts), "rollout_steps_per_launch": steps,
            "obstacle_pairs": {"evaluated": pairs_per_launch, "all": all_pairs},
            "method_tflops": flop / (ms_b * 1e-3) / 1e12,
            "frac_of_fp32_peak": flop / (ms_b * 1e-3) / 1e12 / fp32_peak_tflops(),
            "batched_graph": {"ms_per_launch": ms_b, "rollout_steps_per_s": steps / (ms_b * 1e-3),
                              "solves_per_s": len(insts) / (ms_b * 1e-3)},
            "plain_sequential": {"ms_total": ms_p, "rollout_steps_per_s": steps / (ms_p * 1e-3),
                                 "solves_per_s": len(insts) / (ms_p * 1e-3)}}


def run_stress(reps=3):
    """K=262144, N=200, dt=0.005, 512 spheres + 512 pillars: one solve per
    repetition on device buffers."""
    import torch
    from paper_2407_09812_gb300 import inputs as I
    from paper_2407_09812_gb300 import mppi
    dev = torch.device("cuda")
    prob = I.stress_line()
    K, N, M = prob["params"]["K"], prob["params"]["N"], prob["obstacles"].shape[0]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    x, r, o, u = t(prob["x_hat"]), t(prob["ref"]), t(prob["obstacles"]), t(prob["u_nom"])
    u_out = torch.zeros(N, 4, device=dev)
    s = mppi.Solver(prob["model"], prob["params"])
    pairs = torch.zeros(1, dtype=torch.int64, device=dev)
    s.set_counters(pairs)
    s.solve_async(x, r, o, u, 0, u_out=u_out)
    torch.cuda.synchronize()
    n_pairs = int(pairs.item())
    s.set_counters(None)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(reps):
        s.solve_async(x, r, o, u, i, u_out=u_out)
    e1.record()
    torch.cuda.synchronize()
    s.close()
    ms = e0.elapsed_time(e1) / reps
    flop = K * N * FLOP_PER_STEP + n_pairs * FLOP_PER_PAIR
    return {"workload": "K=262144, N=200, dt=0.005, 512 spheres + 512 vertical cylinders, 12 m/s line",
            "ms_per_solve": ms, "rollout_steps_per_s": K * N / (ms * 1e-3),
            "obstacle_pairs": {"evaluated": n_pairs, "all": K * (N + 1) * M},
            "method_tflops": flop / (ms * 1e-3) / 1e12, "frac_of_fp32_peak": flop / (ms * 1e-3) / 1e12 / fp32_peak_tflops()}


def run_paper_point(reps=50):
    """The paper's own operating point (Table II): K=896, N=15, dt=0.1 s,
    lambda=1e-4, Sigma=diag(0.60, 0.15, 0.15, 0.05) read as a covariance
    (sigma = its square root), Table II weights, motor limits; hover at an
    offset on the figure eight.  The paper runs it in < 10 ms per iteration
    on a Jetson Orin Nano (Sec. IV-A)."""
    import torch
    from paper_2407_09812_gb300 import inputs as I
    from paper_2407_09812_gb300 import mppi
    dev = torch.device("cuda")
    prob = I.paper_operating_point()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    x, r, u = t(prob["x_hat"]), t(prob["ref"]), t(prob["u_nom"])
    uo = torch.zeros(15, 4, device=dev)
    s = mppi.Solver(prob["model"], prob["params"])
    for i in range(5):
        s.solve_async(x, r, None, u, i, u_out=uo)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(reps):
        s.solve_async(x, r, None, u, i, u_out=uo)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    s.close()
    return {"workload": "paper's operating point: K=896, N=15, dt=0.1 s, lambda=1e-4, Table II weights",
            "ms_per_solve": ms, "rollout_steps_per_s": 896 * 15 / (ms * 1e-3),
            "paper": {"ms_per_iteration": "< 10", "rollout_steps_per_s": ">= 1.344e6",
                      "hardware": "Jetson Orin Nano 8 GB (1024-core Ampere GPU at 625 MHz)"}}


def run_options(reps=30):
    """The headline workload with each extension of the paper's method that
    the kernel implements, one at a time: the exact quaternion angle of
    Eq. quat_angle, control interpolation (Sec. IV-B, shift_alpha = 0.1),
    delay compensation (Sec. IV-E, 5 ms), and the occupancy-grid collision
    module (the 64 spheres rasterised into a 0.1 m voxel grid, 6.5 MB, used
    alone).  Device buffers, L2 flushed before each solve, median of `reps`
    solves timed with CUDA events."""
    import torch
    from paper_2407_09812_gb300 import mppi
    dev = torch.device("cuda")
    prob = headline_problem(0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    x, r, u, o = t(prob["x_hat"]), t(prob["ref"]), t(prob["u_nom"]), t(prob["obstacles"])
    u_out = torch.zeros(N_HEAD, 4, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # Occupancy grid of the same spheres (inflated by nothing: the grid marks
    # the obstacles' own volume), 0.1 m voxels over the obstacle box.
    voxel, origin = 0.1, np.array([-21.0, -11.0, -1.0])
    shape = (70, 220, 420)  # (z, y, x)
    centres = [origin[a] + voxel * (np.arange(n) + 0.5) for a, n in ((2, shape[0]), (1, shape[1]), (0, shape[2]))]
    occ = np.zeros(shape, np.uint8)
    for c in prob["obstacles"]:
        lo = [max(0, int((c[a] - c[3] - origin[a]) / voxel)) for a in (2, 1, 0)]
        hi = [min(n, int((c[a] + c[3] - origin[a]) / voxel) + 2) for a, n in zip((2, 1, 0), shape)]
        zc, yc, xc = (centres[i][lo[i]:hi[i]] for i in range(3))
        d2 = ((zc[:, None, None] - c[2]) ** 2 + (yc[None, :, None] - c[1]) ** 2 + (xc[None, None, :] - c[0]) ** 2)
        occ[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] |= (d2 <= c[3] ** 2).astype(np.uint8)
    occ_d = t(occ)
    nz, ny, nx = shape
    variants = [("as configured", {}, None),
                ("exact quaternion angle (Eq. quat_angle)", {"quat_metric": 1}, None),
                ("control interpolation, shift_alpha = 0.1 (Sec. IV-B)", {"shift_alpha": 0.1}, None),
                ("delay compensation, 5 ms (Sec. IV-E)", {"delay": 0.005}, None),
                (f"occupancy grid {nx}x{ny}x{nz} at 0.1 m instead of the spheres", {}, "grid")]
    out = []
    for name, over, mode in variants:
        s = mppi.Solver(prob["model"], dict(prob["params"], **over))
        obs = o
        if mode == "grid":
            s.set_grid(occ_d, tuple(origin), voxel)
            obs = None
        ts = []
        for i in range(reps + 3):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s.solve_async(x, r, obs, u, i, u_out=u_out)
            e1.record()
            torch.cuda.synchronize()
            if i >= 3:
                ts.append(e0.elapsed_time(e1))
        s.close()
        ms = float(np.median(ts))
        entry = {"variant": name, "ms_per_solve": ms, "rollout_steps_per_s": K_HEAD * N_HEAD / (ms * 1e-3)}
        if mode == "grid":
            lookups = K_HEAD * (N_HEAD + 1)
            entry["grid"] = {"bytes": int(occ.size), "lookups_per_solve": lookups,
                             "lookup_bytes_per_s": lookups / (ms * 1e-3),
                             "note": "one 1-byte voxel read per state; the grid fits in L2"}
        out.append(entry)
    return {"workload": WORKLOAD, "variants": out}


def run_serving(args):
    """1000 vehicles at 100 Hz (about 100k requests/s offered, far above one
    GPU's capacity) plus lighter fleets that show the latency below
    saturation."""
    from paper_2407_09812_gb300 import serve
    main = serve.run_fleet(duration_s=args.serve_seconds, n_vehicles=args.serve_vehicles)
    sweep = []
    for nv in (1, 10, 100, 300):
        r = serve.run_fleet(duration_s=max(1.0, min(10.0, args.serve_seconds / 3)), n_vehicles=nv, warmup_s=0.5)
        sweep.append({k: r[k] for k in ("workload", "solves_per_s", "rollout_steps_per_s", "latency_ms",
                                        "missed_ticks", "ticks", "mean_batch")})
    main["lighter_fleets"] = sweep
    return main


def cpu_baseline(seconds: float):
    """The FP64 oracle as it stands, OpenMP over all host cores, on solves
    of the headline workload until about `seconds` have passed."""
    from oracle import oracle as O
    prob = headline_problem(0)
    refs = reference_windows(64)
    threads = os.cpu_count() or 1
    n, t0 = 0, time.perf_counter()
    x, u = prob["x_hat"], prob["u_nom"]
    while True:
        step = dict(prob, x_hat=x, u_nom=u, ref=refs[n % 64], iter=n)
        r = O.mppi_step(step, n_threads=threads)
        x, u = r["x_next"].astype(np.float32), r["u_next"].astype(np.float32)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or n >= 1024:
            break
    rate = K_HEAD * N_HEAD * n / el
    # The same oracle on one core, on a K-subsample of one solve (rollouts
    # are independent, so rollout-steps/s scale with the sample count).
    k1 = 1024
    sub = dict(prob, params=dict(prob["params"], K=k1), ref=refs[0], iter=0)
    t1 = time.perf_counter()
    O.mppi_step(sub, n_threads=1)
    el1 = time.perf_counter() - t1
    rate1 = k1 * N_HEAD / el1
    return {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} full solves of the headline workload (K=16384, N=100, 64 spheres) in {el:.1f} s",
            "solves_per_s": n / el,
            "single_core": {"value": rate1, "unit": UNIT, "cores": 1,
                            "sample": f"one solve of the headline workload with K subsampled to {k1} "
                                      f"in {el1:.2f} s"},
            "parallel_speedup": rate / rate1}


def reference_arm(args) -> dict:
    """The FP64 oracle as it stands, OpenMP over all host cores, as the
    reference arm: the headline closed loop, W untimed and K timed steps,
    each step one solve.  A solve is a bounded sample of the workload: when
    K + W full solves would take more than about 150 s on this host, every
    step solves the first k of the K=16384 samples instead (rollouts are
    independent, so rollout-steps/s carry over), k stated in `sample`."""
    from oracle import oracle as O
    prob = headline_problem(0)
    n_total = args.warmup + args.steps
    refs = reference_windows(n_total)
    threads = os.cpu_count() or 1
    t_all = time.perf_counter()
    x, u = prob["x_hat"], prob["u_nom"]
    # One full solve to size the sample.
    t0 = time.perf_counter()
    r = O.mppi_step(dict(prob, ref=refs[0], iter=0), n_threads=threads)
    t_full = time.perf_counter() - t0
    k = K_HEAD
    if t_full * n_total > 150.0:
        k = max(256, int(K_HEAD * 150.0 / (t_full * n_total)) // 256 * 256)
    params = dict(prob["params"], K=k)
    times = []
    for i in range(n_total):
        step = dict(prob, params=params, x_hat=x, u_nom=u, ref=refs[i], iter=i)
        t0 = time.perf_counter()
        r = O.mppi_step(step, n_threads=threads)
        dt = time.perf_counter() - t0
        x, u = r["x_next"].astype(np.float32), r["u_next"].astype(np.float32)
        if i >= args.warmup:
            times.append(dt)
    times = np.array(times)
    value = k * N_HEAD / float(times.mean())
    sample = (f"{args.steps} timed closed-loop steps of the headline workload, each one solve with "
              f"{'all ' if k == K_HEAD else 'the first '}{k} of the 16384 samples, after {args.warmup} untimed")
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(times.mean() * 1e3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "K": K_HEAD, "N": N_HEAD, "M": M_HEAD},
            "impl": "reference",
            "latency_ms": {"p50": float(np.percentile(times, 50) * 1e3),
                           "p99": float(np.percentile(times, 99) * 1e3)},
            "cpu_baseline": {"kind": "oracle", "cores": threads, "sample": sample, "value": value, "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_all}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-vehicles", type=int, default=1000)
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and serving sections")
    ap.add_argument("--section", default="all", choices=["all", "batched", "stress", "serving", "paper", "options"],
                    help="run one extra section alone and print its JSON (profiling aid)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup(args.gpus)
    args.world = world

    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(reference_arm(args)), flush=True)
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_2407_09812_gb300 import build as B
    B.build()

    if args.section != "all":
        fn = {"batched": lambda: run_batched(args), "stress": run_stress, "serving": lambda: run_serving(args),
              "paper": run_paper_point, "options": run_options}
        print(json.dumps({"section": args.section, **fn[args.section]()}), flush=True)
        return

    res = run_closed_loop(args, rank)
    ms = res["ms"]
    total_ms = float(ms.sum())
    total_ms_max = barrier_max(total_ms, world)
    per_step = total_ms_max / args.steps
    steps_per_solve = K_HEAD * N_HEAD
    value = whole_job_rate(steps_per_solve, args.steps, total_ms_max, world)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    flop_launch = steps_per_solve * FLOP_PER_STEP + res["pairs_per_solve"] * FLOP_PER_PAIR
    achieved = flop_launch / (float(ms.mean()) * 1e-3) / 1e12
    peak = fp32_peak_tflops()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "K": K_HEAD, "N": N_HEAD, "M": M_HEAD, "dt": DT_HEAD,
                   "l2": "flushed between timed steps (256 MiB write outside the step's events)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "solves_per_s": world * args.steps / (total_ms_max * 1e-3),
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                       "mean": float(ms.mean())},
        "gpu_launches": args.steps,
        "clocks": res["clocks"],
        "status_last_step": res["status"],
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": HEADLINE_TRAFFIC_BYTES,
                     "traffic_unit": "bytes per launch (ncu capture)",
                     "kernel": "mppi_step_kernel",
                     "work": {"flop_per_rollout_step": FLOP_PER_STEP, "flop_per_obstacle_pair": FLOP_PER_PAIR,
                              "obstacle_pairs_evaluated_per_solve": res["pairs_per_solve"],
                              "obstacle_pairs_all_per_solve": K_HEAD * (N_HEAD + 1) * M_HEAD},
                     "peak_note": "FP32 FMA peak from unit counts: 152 SMs x 128 lanes x 2 flop x 2070 MHz"},
    }
    line["e2e"] = run_e2e(args, rank, n_steps=min(args.steps, 100))
    if not args.no_extras:
        line["batched"] = run_batched(args)
        line["stress"] = run_stress()
        line["paper_operating_point"] = run_paper_point()
        line["options"] = run_options()
        try:
            line["serving"] = run_serving(args)
        except (ImportError, AttributeError, OSError) as e:
            line["serving"] = {"unavailable": str(e)[:200]}
    line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
