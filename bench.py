"""Benchmark of the MPPI step on GB300: batched vs plain.

Headline workload (one "step" = one control step of a fleet): 256
independent vehicles with uneven problem sizes (K log-uniform in [1024,
32768], N uniform in [30, 150], dt = 0.01 s, 0-128 spheres each, own seeded
initial state and figure-eight phase) solved in ONE persistent launch of the
fused MPPI kernel replayed from a CUDA graph, with the launch shape picked by
the project's batch autotuner.  The fleet runs closed loop on device-resident
inputs: every step each vehicle's warm start is the previous step's shifted
nominal, its state the previous step's plant state, its reference window
advances by dt and its Philox counter by one.

Printed: one JSON line with rollout-steps/s (sum of K*N per second), solves/s
and p50/p99 launch latency; an end-to-end figure through the host-buffer
batched C ABI (mppi_solve_batch_host); the roofline of the batched kernel
against FP32 FMA and MUFU rates measured in the same run; the CPU oracle
timed on the host cores on the same instances; and, as sub-keys, the plain
single-instance paths (the plain step, the same 256 vehicles one launch
each), the single-vehicle closed loop with obstacles, the large-scale stress
solve with its FP64-oracle error, the paper's operating point, the method's
options, the serving loop, and the SM clocks seen while the GPU worked.

`--impl reference` times the FP64 CPU oracle on the same instances instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
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
N_FLEET, FLEET_SEED, FLEET_DT = 256, 2, 0.01
WORKLOAD = ("batched uneven fleet: 256 vehicles, K log-uniform [1024, 32768], N uniform [30, 150], "
            "dt=0.01 s, 0-128 spheres each, own initial state and figure-eight phase; one persistent "
            "launch per control step under CUDA-graph replay, closed loop")
K_HEAD, N_HEAD, DT_HEAD, M_HEAD = 16384, 100, 0.01, 64
CLOSED_LOOP = ("closed-loop figure-eight tracking, K=16384, N=100, dt=0.01 s, 64 spheres, "
               "per-motor thrust limits, lambda=1")

# Algorithmic work, counted from the equations of the method as the oracle
# writes them.  FP32 per rollout step: noise 24, perturb + clamp 12, input
# and rate cost 27, constraint pipeline 95, RK4 437, renormalisation 12,
# tracking cost 43; per evaluated (state, obstacle) pair 17.  MUFU per
# rollout step: Box-Muller 2 lg2, 2 square roots (as rsqrt), 2 sin, 2 cos;
# renormalisation 1 rsqrt; per evaluated pair 1 ex2.  Pairs whose barrier
# term is below its floor (2^-48 of c_bar, where it counts as zero) and that
# cannot be in collision are not part of the result and are not counted;
# the kernel reports how many pairs it evaluated (mppi_set_counters).
FLOP_PER_STEP = 650
FLOP_PER_PAIR = 17
# The counting launch runs one thread per sample (each warp culls with the
# box of its 32 samples' positions, the finest culling of any shape), so the
# work counted does not depend on the shape that is timed: two samples per
# thread cull with a box over 64 positions and evaluate a few more pairs
# that add exactly zero.
COUNT_SHAPE = (128, 1, 0)
MUFU_PER_STEP = {"lg2_ops": 2, "rsqrt_ops": 3, "sin_ops": 2, "cos_ops": 2}
MUFU_PER_PAIR = {"ex2_ops": 1}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the kernel in an ncu capture of the named workload, valid only for the
# kernel source it was taken with (sha256 of the kernel file and its header,
# first 16 hex digits); any other source reports null.
TRAFFIC_CAPTURES = {
    "fleet": {"kernel_sha": "245671fd48323a82", "bytes": 2146048},
    "closed_loop": {"kernel_sha": "245671fd48323a82", "bytes": 118272},
    "stress": {"kernel_sha": "245671fd48323a82", "bytes": 120064},
}
KERNEL_FILES = ("paper_2407_09812_gb300/csrc/mppi_kernels.cu", "paper_2407_09812_gb300/csrc/mppi_internal.h")


def kernel_sha() -> str:
    h = hashlib.sha256()
    for f in KERNEL_FILES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(workload: str):
    c = TRAFFIC_CAPTURES.get(workload)
    if c and c["kernel_sha"] == kernel_sha():
        return c["bytes"]
    return None


# ---------------------------------------------------------------- helpers

class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons, sampled every LOOP_MS ms
    from before the first GPU section to the end of the last one; each
    sample carries the host time it arrived, so a section's share can be
    picked (20 ms: a few samples fall inside even a 20-step timed region of
    the headline, 90 ms long)."""

    LOOP_MS = 20

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.samples = []  # (host time, sm MHz, max MHz, power W, reasons)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.LOOP_MS)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            t0 = time.time()
            while not self.samples and time.time() - t0 < 5.0:
                time.sleep(0.01)
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            p = [x.strip() for x in line.strip().split(",")]
            if len(p) < 9:
                continue
            try:
                sm, mx = float(p[1]), float(p[2])
                pw = float(p[3]) if p[3].replace(".", "", 1).isdigit() else float("nan")
            except ValueError:
                continue
            reasons = {n for n, v in zip(self.NAMES, p[5:9]) if v.lower() == "active"}
            self.samples.append((time.perf_counter(), sm, mx, pw, reasons))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0=None, t1=None) -> dict:
        sel = [s for s in self.samples if (t0 is None or s[0] >= t0) and (t1 is None or s[0] <= t1)]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = set().union(*[s[4] for s in sel])
        return {"sm_mhz": float(np.median([s[1] for s in sel])), "sm_max_mhz": float(max(s[2] for s in sel)),
                "reasons": sorted(reasons), "samples": len(sel),
                "power_w_max": float(np.nanmax([s[3] for s in sel]))}


def dist_setup():
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
    (replicas: every rank solves its own fleet; weak scaling)."""
    return world * units_per_step_per_rank * steps / (max_ms * 1e-3)


def roofline(flop: float, mufu: dict, ms: float, peaks: dict, traffic, what: str) -> dict:
    """FP32 and MUFU fractions of one launch of `ms` milliseconds against
    the rates measured in this run."""
    achieved = flop / (ms * 1e-3) / 1e12
    peak = peaks["fp32_flops"] / 1e12
    mufu_s = sum(n / peaks[op] for op, n in mufu.items())
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_unit": "DRAM bytes per launch (ncu capture of this kernel source)",
            "kernel": f"mppi_step_kernel ({what})",
            "peak_source": "of measured: FFMA micro-benchmark (mppi_measure_peaks) in this run",
            "mufu": {"ops_per_launch": float(sum(mufu.values())), "frac": mufu_s / (ms * 1e-3),
                     "note": "time the launch's MUFU work needs at the measured MUFU rates / launch time"}}


def mufu_ops(rollout_steps: float, pairs: float) -> dict:
    out = {op: rollout_steps * n for op, n in MUFU_PER_STEP.items()}
    for op, n in MUFU_PER_PAIR.items():
        out[op] = out.get(op, 0.0) + pairs * n
    return out


def shape_dict(s) -> dict:
    return {"block": s[0], "lanes": s[1], "pipelined": s[2], "list_margin": s[3],
            "samples_per_thread": s[4] if len(s) > 4 else 1}


def flusher():
    import torch
    return torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2


# ------------------------------------------------------------- the fleet

class Fleet:
    """The headline workload's 256 vehicles laid out for the batched entry
    points: every per-vehicle array is a slice of one flat array (device or
    host), so a step's descriptors are updated with vectorised operations.
    The reference of vehicle i is one long sampled trajectory; the window
    of step t starts 13 t floats in."""

    def __init__(self, n_steps: int, stream_base: int = 0):
        from paper_2407_09812_gb300 import inputs as I
        self.probs = I.batched_uneven(n=N_FLEET, seed=FLEET_SEED, dt=FLEET_DT)
        for i, p in enumerate(self.probs):
            p["params"] = dict(p["params"], stream_id=stream_base + i)
        self.n = len(self.probs)
        self.K = np.array([p["params"]["K"] for p in self.probs], np.int64)
        self.N = np.array([p["params"]["N"] for p in self.probs], np.int64)
        self.M = np.array([p["obstacles"].shape[0] for p in self.probs], np.int64)
        self.rollout_steps = int((self.K * self.N).sum())
        self.n_steps = n_steps
        # Flat layouts (float offsets; every segment a multiple of 4 floats).
        self.rlen = 13 * (n_steps + self.N + 1)
        self.roff = np.concatenate([[0], np.cumsum((self.rlen + 3) // 4 * 4)[:-1]])
        self.uoff = np.concatenate([[0], np.cumsum(4 * self.N)[:-1]])
        self.ooff = np.concatenate([[0], np.cumsum(4 * self.M)[:-1]])
        ref = np.zeros(int(((self.rlen + 3) // 4 * 4).sum()), np.float32)
        for i, p in enumerate(self.probs):
            traj = I.Trajectory("eight", {"phase": p["phase"]})
            w = traj.window(0.0, int(n_steps + self.N[i]), FLEET_DT)
            ref[self.roff[i]:self.roff[i] + w.size] = w.reshape(-1)
        self.ref = ref
        self.obs = np.concatenate([p["obstacles"].reshape(-1) for p in self.probs]).astype(np.float32)
        self.x0 = np.zeros((self.n, 16), np.float32)
        self.u0 = np.concatenate([p["u_nom"].reshape(-1) for p in self.probs]).astype(np.float32)
        for i, p in enumerate(self.probs):
            self.x0[i, :13] = p["x_hat"]
        self.iter0 = np.array([p["iter"] for p in self.probs], np.uint64)

    def records(self, INSTANCE_DTYPE, base: dict, ping: int) -> np.ndarray:
        """Descriptors of one ping-pong phase: state and nominal read from
        buffer `ping`, warm start and plant state written to the other.
        `base` holds the flat arrays' addresses."""
        r = np.zeros(self.n, INSTANCE_DTYPE)
        a, b = ping, 1 - ping
        r["x_hat"] = base["x"][a] + 64 * np.arange(self.n)
        r["x_next"] = base["x"][b] + 64 * np.arange(self.n)
        r["u_nom"] = base["u"][a] + 4 * self.uoff
        r["u_next"] = base["u"][b] + 4 * self.uoff
        r["u_out"] = base["u_out"] + 4 * self.uoff
        r["u_cmd"] = base["u_cmd"] + 16 * np.arange(self.n)
        r["status"] = base["status"] + 4 * np.arange(self.n)
        r["obstacles"] = np.where(self.M > 0, base["obs"] + 4 * self.ooff, 0)
        r["ref"] = base["ref"] + 4 * self.roff
        r["iter"] = self.iter0
        r["K"], r["N"], r["M"] = self.K, self.N, self.M
        for i, p in enumerate(self.probs):
            q = p["params"]
            r["dt"][i], r["lam"][i], r["sigma"][i] = q["dt"], q["lambda"], q["sigma"]
            r["seed"][i], r["stream_id"][i] = q["seed"], q["stream_id"]
        return r

    def device_buffers(self):
        import torch
        dev = torch.device("cuda")
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        b = {"x": [t(self.x0), t(self.x0)], "u": [t(self.u0), t(self.u0)], "ref": t(self.ref),
             "obs": t(self.obs) if self.obs.size else torch.zeros(4, device=dev),
             "u_out": torch.zeros(self.u0.size, device=dev), "u_cmd": torch.zeros(self.n, 4, device=dev),
             "status": torch.zeros(self.n, dtype=torch.int32, device=dev)}
        addr = {k: ([v[0].data_ptr(), v[1].data_ptr()] if isinstance(v, list) else v.data_ptr())
                for k, v in b.items()}
        return b, addr

    def host_buffers(self):
        import torch
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        b = {"x": [pin(self.x0), pin(self.x0)], "u": [pin(self.u0), pin(self.u0)], "ref": pin(self.ref),
             "obs": pin(self.obs if self.obs.size else np.zeros(4, np.float32)),
             "u_out": pin(np.zeros(self.u0.size, np.float32)), "u_cmd": pin(np.zeros((self.n, 4), np.float32)),
             "status": pin(np.zeros(self.n, np.int32))}
        addr = {k: ([v[0].ctypes.data, v[1].ctypes.data] if isinstance(v, list) else v.ctypes.data)
                for k, v in b.items()}
        return b, addr

    def dicts(self, bufs, ping=0):
        """The fleet as per-instance dicts of torch tensors (for the tuner and
        the one-by-one launches), sharing the flat device buffers."""
        out = []
        a = ping
        for i, p in enumerate(self.probs):
            N, M, u0 = int(self.N[i]), int(self.M[i]), int(self.uoff[i])
            q = p["params"]
            out.append({"x_hat": bufs["x"][a][i, :13], "ref": bufs["ref"][self.roff[i]:self.roff[i] + 13 * (N + 1)],
                        "obstacles": bufs["obs"][self.ooff[i]:self.ooff[i] + 4 * M] if M else None,
                        "u_nom": bufs["u"][a][u0:u0 + 4 * N], "u_out": bufs["u_out"][u0:u0 + 4 * N],
                        "u_cmd": bufs["u_cmd"][i], "K": int(self.K[i]), "N": N, "dt": q["dt"],
                        "lambda": q["lambda"], "sigma": q["sigma"], "seed": q["seed"], "stream_id": q["stream_id"],
                        "iter": int(self.iter0[i])})
        return out

    def h2d_d2h_bytes(self):
        """Bytes of mppi_solve_batch_host's two copies (16-byte segments)."""
        up4 = lambda v: (v + 3) // 4 * 4
        h2d = 4 * int((16 + up4(13 * (self.N + 1)) + 4 * self.M + 4 * self.N).sum())
        d2h = 4 * int((8 * self.N + 24).sum())
        return h2d, d2h


def run_fleet(args, rank: int, peaks: dict, clk: ClockSampler):
    """The headline: batch-autotuned shape, then W untimed and K timed
    closed-loop steps, one graph-replayed persistent launch each, timed
    with CUDA events on the launching stream; the L2 is flushed between
    steps outside the events."""
    import torch
    from paper_2407_09812_gb300 import mppi
    n_total = args.warmup + args.steps
    fleet = Fleet(n_total, stream_base=rank * N_FLEET)
    bufs, addr = fleet.device_buffers()
    rec = [fleet.records(mppi.INSTANCE_DTYPE, addr, 0), fleet.records(mppi.INSTANCE_DTYPE, addr, 1)]
    cap = {"max_instances": fleet.n, "max_samples": int(fleet.K.sum()), "N_max": int(fleet.N.max()),
           "M_max": int(max(1, fleet.M.max()))}
    p0 = fleet.probs[0]
    solver = mppi.Solver(p0["model"], p0["params"], cap)
    stream = torch.cuda.current_stream()
    t_tune = time.perf_counter()
    if args.shape:
        shape = tuple(float(v) if i == 3 else int(v) for i, v in enumerate(args.shape.split(",")))
        solver.set_shape(*shape)
    else:
        shape = solver.autotune_batch(fleet.dicts(bufs), stream=stream)
    t_tune = time.perf_counter() - t_tune
    pairs = torch.zeros(1, dtype=torch.int64, device="cuda")
    solver.set_shape(*COUNT_SHAPE)
    solver.set_counters(pairs)  # evaluated obstacle pairs of step 0, in an untimed launch
    solver.solve_batch(rec[0], stream=stream, graph=False)
    torch.cuda.synchronize()
    pairs_per_launch = int(pairs.item())
    solver.set_counters(None)
    if args.shape:
        solver.set_shape(*shape)
    else:
        solver.set_shape(0, 0, 0)  # back to the tuned shape
    flush = flusher()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_total)]

    def step(i):
        r = rec[i % 2]
        r["ref"] = addr["ref"] + 4 * fleet.roff + 52 * i
        r["iter"] = fleet.iter0 + np.uint64(i)
        solver.solve_batch(r, stream=stream, graph=True)

    for i in range(args.warmup):
        flush.zero_()
        step(i)
    torch.cuda.synchronize()
    barrier(args.world)
    t0 = time.perf_counter()
    for i in range(args.warmup, n_total):
        flush.zero_()
        ev[i][0].record(stream)
        step(i)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    barrier(args.world)
    ms = np.array([ev[i][0].elapsed_time(ev[i][1]) for i in range(args.warmup, n_total)])
    status = bufs["status"].cpu().numpy()
    final_x = bufs["x"][n_total % 2].cpu().numpy()
    solver.close()
    return {"ms": ms, "fleet": fleet, "shape": shape, "tune_s": t_tune, "pairs": pairs_per_launch,
            "status_ok": int((status == 0).sum()), "finite": bool(np.all(np.isfinite(final_x))),
            "window": (t0, t1)}


def run_fleet_e2e(args, fleet: Fleet, shape, n_steps: int):
    """The same closed loop through mppi_solve_batch_host with HOST buffers
    (pinned): every step packs the fleet's inputs, copies them in, solves,
    copies the outputs back and unpacks them."""
    from paper_2407_09812_gb300 import mppi
    bufs, addr = fleet.host_buffers()
    rec = [fleet.records(mppi.INSTANCE_DTYPE, addr, 0), fleet.records(mppi.INSTANCE_DTYPE, addr, 1)]
    p0 = fleet.probs[0]
    cap = {"max_instances": fleet.n, "max_samples": int(fleet.K.sum()), "N_max": int(fleet.N.max()),
           "M_max": int(max(1, fleet.M.max()))}
    solver = mppi.Solver(p0["model"], p0["params"], cap)
    solver.set_shape(*shape)
    lat = []
    for i in range(n_steps + 3):
        r = rec[i % 2]
        r["ref"] = addr["ref"] + 4 * fleet.roff + 52 * i
        r["iter"] = fleet.iter0 + np.uint64(i)
        t0 = time.perf_counter()
        solver.solve_batch_host(r)
        dt = time.perf_counter() - t0
        if i >= 3:
            lat.append(dt)
    solver.close()
    lat = np.array(lat)
    h2d, d2h = fleet.h2d_d2h_bytes()
    return {"value": fleet.rollout_steps / float(lat.mean()), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": float(lat.mean() * 1e3),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "solves_per_s": fleet.n / float(lat.mean()),
            "api": "mppi_solve_batch_host (host buffers, one packed copy each way, synchronous)"}


def run_one_by_one(fleet: Fleet):
    """The same 256 instances, one single-instance launch each (the plain
    path), device buffers, each launch with the handle's default shape."""
    import torch
    from paper_2407_09812_gb300 import mppi
    bufs, _ = fleet.device_buffers()
    insts = fleet.dicts(bufs)
    plain = mppi.Solver(fleet.probs[0]["model"], fleet.probs[0]["params"],
                        {"max_instances": 1, "max_samples": 32768, "N_max": 150, "M_max": 128})
    stream = torch.cuda.current_stream()
    flush = flusher()

    def one_pass():
        for p, d in zip(fleet.probs, insts):
            plain.set_params(p["params"])
            plain.solve_async(d["x_hat"], d["ref"], d["obstacles"], d["u_nom"], d["iter"], u_out=d["u_out"],
                              u_cmd=d["u_cmd"], stream=stream)

    one_pass()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(3):
        flush.zero_()
        e0.record(stream)
        one_pass()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    plain.close()
    ms = float(np.median(times))
    return {"workload": "the same 256 instances, one single-instance launch each (default shapes)",
            "ms_total": ms, "rollout_steps_per_s": fleet.rollout_steps / (ms * 1e-3),
            "solves_per_s": fleet.n / (ms * 1e-3)}


def run_plain_step(reps=30):
    """The plain single MPPI step: K=1024, N=50, dt=0.02, hover reference,
    0.5 m offset, box-clamped inputs, no obstacles; device buffers, L2
    flushed before each solve, CUDA events per solve."""
    import torch
    from paper_2407_09812_gb300 import inputs as I
    from paper_2407_09812_gb300 import mppi
    prob = I.plain_hover()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x, r, u = t(prob["x_hat"]), t(prob["ref"]), t(prob["u_nom"])
    uo = torch.zeros(50, 4, device="cuda")
    s = mppi.Solver(prob["model"], prob["params"])
    flush = flusher()
    ts = []
    for i in range(reps + 3):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.solve_async(x, r, None, u, i, u_out=uo)
        e1.record()
        torch.cuda.synchronize()
        if i >= 3:
            ts.append(e0.elapsed_time(e1))
    shape = s.get_shape(1024, 50, 0)
    s.close()
    ts = np.array(ts)
    return {"workload": "plain step: K=1024, N=50, dt=0.02 s, hover reference, 0.5 m offset, box clamp, no obstacles",
            "ms_per_solve": float(np.median(ts)), "p99_ms": float(np.percentile(ts, 99)),
            "rollout_steps_per_s": 1024 * 50 / (float(np.median(ts)) * 1e-3),
            "solves_per_s": 1e3 / float(np.median(ts)), "shape": shape_dict(shape)}


# -------------------------------------------- single-vehicle closed loop

def headline_problem(rank: int = 0):
    from paper_2407_09812_gb300 import inputs as I
    return I.eight_with_spheres(K=K_HEAD, N=N_HEAD, dt=DT_HEAD, M=M_HEAD, seed=1, stream_id=rank)


def reference_windows(n_steps: int):
    from paper_2407_09812_gb300 import inputs as I
    traj = I.Trajectory("eight")
    return np.stack([traj.window(DT_HEAD * t, N_HEAD, DT_HEAD) for t in range(n_steps)])


def run_closed_loop(n_steps: int, peaks: dict, warmup=5, shape=None):
    """One vehicle, K=16384, N=100, 64 spheres: closed loop on device
    buffers, one solve per control step (CUDA events per solve, L2 flushed
    between), then the same loop through mppi_solve with host buffers."""
    import torch
    from paper_2407_09812_gb300 import mppi
    dev = torch.device("cuda")
    prob = headline_problem()
    n_total = warmup + n_steps
    refs_h = reference_windows(n_total)
    refs = torch.from_numpy(refs_h).to(dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    obs = t(prob["obstacles"])
    x = [t(prob["x_hat"]), torch.zeros(13, device=dev)]
    u = [t(prob["u_nom"]), torch.zeros(N_HEAD, 4, device=dev)]
    u_out = torch.zeros(N_HEAD, 4, device=dev)
    u_cmd = torch.zeros(4, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    solver = mppi.Solver(prob["model"], prob["params"])
    if shape:
        solver.set_shape(*shape)
    else:
        shape = solver.autotune_on({"x_hat": x[0], "ref": refs[0], "obstacles": obs, "u_nom": u[0], "K": K_HEAD,
                                    "N": N_HEAD, "dt": DT_HEAD, "lambda": prob["params"]["lambda"],
                                    "sigma": prob["params"]["sigma"], "seed": prob["params"]["seed"], "iter": 0})
    flush = flusher()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_total)]

    def step(i):
        a, b = i % 2, (i + 1) % 2
        solver.solve_async(x[a], refs[i], obs, u[a], i, u_out=u_out, u_cmd=u_cmd, u_next=u[b], x_next=x[b],
                           status=status, stream=stream)

    pairs = torch.zeros(1, dtype=torch.int64, device=dev)
    solver.set_counters(pairs)
    for i in range(warmup):
        flush.zero_()
        step(i)
    torch.cuda.synchronize()
    pairs_per_solve = int(pairs.item()) / warmup
    solver.set_counters(None)
    for i in range(warmup, n_total):
        flush.zero_()
        ev[i][0].record(stream)
        step(i)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = np.array([ev[i][0].elapsed_time(ev[i][1]) for i in range(warmup, n_total)])
    st = int(status.item())
    solver.close()
    # Host buffers through mppi_solve.
    solver = mppi.Solver(prob["model"], prob["params"])
    solver.set_shape(*shape)
    xh, uh = prob["x_hat"].copy(), prob["u_nom"].copy()
    lat = []
    n_e2e = min(n_steps, 100)
    for i in range(n_e2e + 3):
        t0 = time.perf_counter()
        out = solver.solve(xh, refs_h[i % n_total], prob["obstacles"], uh, i)
        dt = time.perf_counter() - t0
        xh, uh = out["x_next"], out["u_next"]
        if i >= 3:
            lat.append(dt)
    solver.close()
    lat = np.array(lat)
    N, M = N_HEAD, M_HEAD
    up4 = lambda v: (v + 3) // 4 * 4
    h2d = 4 * up4(up4(up4(16 + 13 * (N + 1)) + 4 * M) + 4 * N)
    d2h = 4 * (up4(4 * N) + 4 + up4(4 * N) + 16 + 4)
    steps = K_HEAD * N_HEAD
    mean = float(ms.mean())
    return {"workload": CLOSED_LOOP, "steps": n_steps, "shape": shape_dict(shape),
            "ms_per_solve": mean, "rollout_steps_per_s": steps / (mean * 1e-3), "solves_per_s": 1e3 / mean,
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
            "status_last_step": st,
            "roofline": roofline(steps * FLOP_PER_STEP + pairs_per_solve * FLOP_PER_PAIR,
                                 mufu_ops(steps, pairs_per_solve), mean, peaks, captured_traffic("closed_loop"),
                                 "single instance"),
            "obstacle_pairs": {"evaluated": pairs_per_solve, "all": K_HEAD * (N_HEAD + 1) * M_HEAD},
            "e2e": {"value": steps / float(lat.mean()), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": float(lat.mean() * 1e3),
                    "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                    "api": "mppi_solve (host buffers, synchronous)"}}


# ----------------------------------------------------------------- stress

def run_stress(peaks: dict, reps=3, shape=None):
    """K=262144, N=200, dt=0.005, 512 spheres + 512 pillars: one solve per
    repetition on device buffers with the instance-autotuned shape; the
    outputs of the last solve are kept for the oracle comparison."""
    import torch
    from paper_2407_09812_gb300 import inputs as I
    from paper_2407_09812_gb300 import mppi
    dev = torch.device("cuda")
    prob = I.stress_line()
    K, N, M = prob["params"]["K"], prob["params"]["N"], prob["obstacles"].shape[0]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    x, r, o, u = t(prob["x_hat"]), t(prob["ref"]), t(prob["obstacles"]), t(prob["u_nom"])
    out = {k: torch.zeros(n, device=dev) for k, n in (("u_out", (N, 4)), ("u_cmd", 4), ("u_next", (N, 4)),
                                                       ("x_next", 13), ("costs", K))}
    s = mppi.Solver(prob["model"], prob["params"])
    if shape:
        s.set_shape(*shape)
    else:
        shape = s.autotune_on({"x_hat": x, "ref": r, "obstacles": o, "u_nom": u, "K": K, "N": N,
                               "dt": prob["params"]["dt"], "lambda": prob["params"]["lambda"],
                               "sigma": prob["params"]["sigma"], "seed": prob["params"]["seed"], "iter": 0})
    pairs = torch.zeros(1, dtype=torch.int64, device=dev)
    s.set_shape(*COUNT_SHAPE)
    s.set_counters(pairs)
    s.solve_async(x, r, o, u, prob["iter"], u_out=out["u_out"])
    torch.cuda.synchronize()
    n_pairs = int(pairs.item())
    s.set_counters(None)
    s.set_shape(*shape)
    flush = flusher()
    ts = []
    for i in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.solve_async(x, r, o, u, prob["iter"], **out)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    s.close()
    ms = float(np.median(ts))
    steps = K * N
    res = {"workload": "K=262144, N=200, dt=0.005, 512 spheres + 512 vertical cylinders, 12 m/s line",
           "shape": shape_dict(shape), "ms_per_solve": ms, "rollout_steps_per_s": steps / (ms * 1e-3),
           "obstacle_pairs": {"evaluated": n_pairs, "all": K * (N + 1) * M},
           "roofline": roofline(steps * FLOP_PER_STEP + n_pairs * FLOP_PER_PAIR, mufu_ops(steps, n_pairs), ms,
                                peaks, captured_traffic("stress"), "single instance")}
    gpu = {k: v.cpu().numpy() for k, v in out.items()}
    return res, prob, gpu


def stress_oracle_error(prob, gpu) -> tuple:
    """The FP64 oracle's full step on the stress problem (all host cores),
    outside every timed region: relative errors of the GPU's update, warm
    start, command and per-sample costs (the update error per control is
    measured against max(|u_oracle|, sigma_c)); the oracle's time is that
    workload's CPU baseline."""
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref = O.mppi_step(prob, n_threads=threads)
    el = time.perf_counter() - t0
    sig = np.asarray(prob["params"]["sigma"], np.float64)

    def uerr(a, b):
        a, b = np.asarray(a, np.float64).reshape(-1, 4), np.asarray(b, np.float64).reshape(-1, 4)
        return float((np.abs(a - b) / np.maximum(np.abs(b), sig[None, :])).max())

    c_orc, c_gpu = ref["costs"], gpu["costs"].astype(np.float64)
    keep = np.isfinite(c_orc) & ~(np.abs(ref["min_gap"]) < 1e-4)
    err = {"update": uerr(gpu["u_out"], ref["u_out"]), "warm_start": uerr(gpu["u_next"], ref["u_next"]),
           "command": uerr(gpu["u_cmd"], ref["u_cmd"]),
           "costs": float((np.abs(c_gpu[keep] - c_orc[keep]) / np.abs(c_orc[keep])).max()),
           "costs_compared": int(keep.sum()), "grazing_excluded": int((~keep).sum()),
           "tolerance": 1e-4, "effective_samples": float(1.0 / np.sum(ref["weights"] ** 2))}
    K, N = prob["params"]["K"], prob["params"]["N"]
    cpu = {"value": K * N / el, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"one full FP64 solve of the stress workload in {el:.1f} s"}
    return err, cpu


# ------------------------------------------------------- other sections

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
    """The single-vehicle closed-loop workload with each extension of the
    paper's method that the kernel implements, one at a time: the exact
    quaternion angle of Eq. quat_angle, control interpolation (Sec. IV-B,
    shift_alpha = 0.1), delay compensation (Sec. IV-E, 5 ms), and the
    occupancy-grid collision module (the 64 spheres rasterised into a 0.1 m
    voxel grid, 6.5 MB, used alone).  Device buffers, L2 flushed before each
    solve, median of `reps` solves timed with CUDA events."""
    import torch
    from paper_2407_09812_gb300 import mppi
    dev = torch.device("cuda")
    prob = headline_problem(0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    x, r, u, o = t(prob["x_hat"]), t(prob["ref"]), t(prob["u_nom"]), t(prob["obstacles"])
    u_out = torch.zeros(N_HEAD, 4, device=dev)
    flush = flusher()
    # Occupancy grid of the same spheres (the obstacles' own volume), 0.1 m
    # voxels over the obstacle box.
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
    return {"workload": CLOSED_LOOP, "variants": out}


def serving_mix_batched(n_vehicles: int, max_batch_samples: int = 1 << 21, reps: int = 3):
    """The serving fleet's vehicles (same K, N, obstacles and references)
    solved as graph-replayed batched launches of at most `max_batch_samples`
    samples each, device buffers, no queue: the throughput serving can reach
    on this mix."""
    import torch
    from paper_2407_09812_gb300 import inputs as I
    from paper_2407_09812_gb300 import mppi
    fleet = I.serving_fleet(n_vehicles=n_vehicles)
    model = I.model(motor_clip=1)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    batches, cur, samples = [], [], 0
    for i, v in enumerate(fleet):
        if cur and samples + v["K"] > max_batch_samples:
            batches.append(cur)
            cur, samples = [], 0
        ref = I.Trajectory("eight", {"phase": v["phase"]}).window(0.0, v["N"], v["dt"])
        cur.append({"x_hat": t(ref[0]), "ref": t(ref), "obstacles": t(v["obstacles"]),
                    "u_nom": t(I.hover_u(model, v["N"])), "u_out": torch.zeros(v["N"], 4, device="cuda"),
                    "K": v["K"], "N": v["N"], "dt": v["dt"], "lambda": 1.0, "sigma": (1.0, 1.0, 1.0, 0.5),
                    "seed": v["seed"], "stream_id": v["stream_id"], "iter": 0})
        samples += v["K"]
    batches.append(cur)
    solver = mppi.Solver(model, I.params(), {"max_instances": max(len(b) for b in batches),
                                            "max_samples": max_batch_samples, "N_max": 100, "M_max": 32})
    for b in batches:
        solver.solve_batch(b, graph=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        for b in batches:
            solver.solve_batch(b, graph=True)
    e1.record()
    torch.cuda.synchronize()
    solver.close()
    s = e0.elapsed_time(e1) * 1e-3 / reps
    steps = sum(v["K"] * v["N"] for v in fleet)
    return {"workload": f"the serving fleet's {n_vehicles} vehicles as {len(batches)} graph-replayed batched "
                        f"launches of <= {max_batch_samples} samples, device buffers",
            "solves_per_s": n_vehicles / s, "rollout_steps_per_s": steps / s}


def run_serving(args):
    """1000 vehicles at 100 Hz (about 100k requests/s offered, far above one
    GPU's capacity) plus lighter fleets that show the latency below
    saturation, and the same mix solved as plain batched launches."""
    from paper_2407_09812_gb300 import serve
    main = serve.run_fleet(duration_s=args.serve_seconds, n_vehicles=args.serve_vehicles)
    main["batched_same_mix"] = serving_mix_batched(args.serve_vehicles)
    sweep = []
    for nv in (1, 10, 100, 300):
        r = serve.run_fleet(duration_s=max(1.0, min(10.0, args.serve_seconds / 3)), n_vehicles=nv, warmup_s=0.5)
        sweep.append({k: r[k] for k in ("workload", "solves_per_s", "rollout_steps_per_s", "latency_ms",
                                        "missed_ticks", "ticks", "mean_batch", "p99_batch") if k in r})
    main["lighter_fleets"] = sweep
    return main


# ------------------------------------------------------------ CPU oracle

def oracle_on_fleet(probs, budget_s: float, threads: int = 0):
    """Solves fleet instances with the FP64 oracle (OpenMP over each
    instance's samples, all host cores unless `threads` is given), in order,
    until `budget_s` has passed (at least one, at most all); returns
    (rollout-steps, solves, seconds)."""
    from oracle import oracle as O
    threads = threads or os.cpu_count() or 1
    steps = n = 0
    t0 = time.perf_counter()
    while True:
        p = probs[n]
        O.mppi_step(p, n_threads=threads)
        steps += p["params"]["K"] * p["params"]["N"]
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n == len(probs):
            return steps, n, el


def host_cpu() -> str:
    """Architecture and CPU model of the host (lscpu, best effort)."""
    import platform
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return f"{platform.machine()}, {model}" if model else platform.machine()


def cpu_baseline(seconds: float):
    """The FP64 oracle as it stands, OpenMP over all host cores, on the
    fleet's instances in order until about `seconds` have passed; rates are
    rollout-steps of the instances solved per second."""
    from paper_2407_09812_gb300 import inputs as I
    probs = I.batched_uneven(n=N_FLEET, seed=FLEET_SEED, dt=FLEET_DT)
    steps, n, el = oracle_on_fleet(probs, seconds)
    # The same on one host thread, on the smallest instances (a shorter
    # sample): the oracle's own per-core rate, for the OpenMP leg's scaling.
    small = sorted(probs, key=lambda p: p["params"]["K"] * p["params"]["N"])
    s1, n1, el1 = oracle_on_fleet(small, max(1.0, seconds / 4), threads=1)
    return {"value": steps / el, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle", "cpu": host_cpu(),
            "sample": f"the first {n} of the 256 fleet instances in order, each one full FP64 solve, in {el:.1f} s",
            "solves_per_s": n / el,
            "single_thread": {"value": s1 / el1, "unit": UNIT, "cores": 1,
                              "sample": f"the {n1} smallest fleet instances (K N), one full FP64 solve each on one "
                                        f"host thread, in {el1:.1f} s"}}


def reference_arm(args) -> dict:
    """The FP64 oracle as it stands, OpenMP over all host cores, as the
    reference arm on the headline fleet: W untimed and K timed steps; each
    step solves a bounded sample of the fleet, the next `per_step`
    instances in order (wrapping), sized from one calibration solve so that
    the whole run takes about `--ref-seconds`; rollout-steps/s are those
    of the instances solved."""
    from paper_2407_09812_gb300 import inputs as I
    probs = I.batched_uneven(n=N_FLEET, seed=FLEET_SEED, dt=FLEET_DT)
    n_total = args.warmup + args.steps
    t_all = time.perf_counter()
    s0, _, e0 = oracle_on_fleet(probs, min(1.0, 0.05 * args.ref_seconds))  # calibration
    rate = s0 / e0
    fleet_steps = sum(p["params"]["K"] * p["params"]["N"] for p in probs)
    fleet_s = fleet_steps / rate
    per_step = int(max(1, min(N_FLEET, N_FLEET * args.ref_seconds / (fleet_s * n_total))))
    times, steps_solved, at = [], [], 0
    for i in range(n_total):
        from oracle import oracle as O
        threads = os.cpu_count() or 1
        t0 = time.perf_counter()
        st = 0
        for j in range(per_step):
            p = probs[(at + j) % N_FLEET]
            O.mppi_step(dict(p, iter=p["iter"] + i), n_threads=threads)
            st += p["params"]["K"] * p["params"]["N"]
        dt = time.perf_counter() - t0
        at = (at + per_step) % N_FLEET
        if i >= args.warmup:
            times.append(dt)
            steps_solved.append(st)
    times = np.array(times)
    value = float(np.sum(steps_solved) / times.sum())
    sample = (f"{args.steps} timed steps after {args.warmup} untimed; each step solves the next {per_step} of the "
              f"256 fleet instances (in order, wrapping), each one full FP64 solve")
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(times.mean() * 1e3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances": N_FLEET},
            "impl": "reference", "solves_per_s": per_step * len(times) / float(times.sum()),
            "latency_ms": {"p50": float(np.percentile(times, 50) * 1e3),
                           "p99": float(np.percentile(times, 99) * 1e3)},
            "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count() or 1, "cpu": host_cpu(), "sample": sample,
                             "value": value, "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_all}


# ------------------------------------------------------------------ main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=150.0, help="reference arm: oracle time for the whole run")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-vehicles", type=int, default=1000)
    ap.add_argument("--no-extras", action="store_true", help="only the headline fleet and its end-to-end figure")
    ap.add_argument("--no-oracle", action="store_true", help="skip the stress workload's FP64 oracle comparison")
    ap.add_argument("--shape", default="", help="launch shape 'block,lanes,pipelined,margin[,samples_per_thread]' instead of the "
                                                "batch autotuner's (profiling aid)")
    ap.add_argument("--section", default="all",
                    choices=["all", "fleet", "closed_loop", "stress", "serving", "paper", "options", "plain"],
                    help="run one section alone and print its JSON (profiling aid)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()
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
    from paper_2407_09812_gb300 import mppi
    clk = ClockSampler(torch.cuda.current_device()).start()
    peaks = mppi.measure_peaks()

    if args.section != "all":
        forced = tuple(float(v) if i == 3 else int(v) for i, v in enumerate(args.shape.split(","))) \
            if args.shape else None
        fn = {"fleet": lambda: run_fleet(args, rank, peaks, clk)["ms"].tolist(),
              "closed_loop": lambda: run_closed_loop(args.steps, peaks, shape=forced),
              "stress": lambda: run_stress(peaks, shape=forced)[0], "serving": lambda: run_serving(args),
              "paper": run_paper_point, "options": run_options, "plain": run_plain_step}
        out = fn[args.section]()
        clk.stop()
        print(json.dumps({"section": args.section, "result": out, "peaks": peaks}), flush=True)
        return

    res = run_fleet(args, rank, peaks, clk)
    fleet = res["fleet"]
    ms = res["ms"]
    total_ms_max = barrier_max(float(ms.sum()), world)
    value = whole_job_rate(fleet.rollout_steps, args.steps, total_ms_max, world)

    if rank != 0:
        clk.stop()
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    mean = float(ms.mean())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances": fleet.n, "rollout_steps_per_launch": fleet.rollout_steps,
                   "sum_K": int(fleet.K.sum()), "N_range": [int(fleet.N.min()), int(fleet.N.max())],
                   "M_range": [int(fleet.M.min()), int(fleet.M.max())],
                   "l2": "flushed between timed steps (256 MiB write outside the step's events)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "solves_per_s": world * fleet.n * args.steps / (total_ms_max * 1e-3),
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)), "mean": mean,
                       "note": "one persistent launch solves all 256 vehicles: a vehicle's solve latency is "
                               "its launch's"},
        "gpu_launches": args.steps,
        "shape": shape_dict(res["shape"]), "autotune_s": res["tune_s"],
        "status_ok_last_step": res["status_ok"], "state_finite": res["finite"],
        "roofline": roofline(fleet.rollout_steps * FLOP_PER_STEP + res["pairs"] * FLOP_PER_PAIR,
                             mufu_ops(fleet.rollout_steps, res["pairs"]), mean, peaks, captured_traffic("fleet"),
                             "batched launch of 256 uneven instances"),
        "obstacle_pairs": {"evaluated_per_launch": res["pairs"],
                           "all_per_launch": int((fleet.K * (fleet.N + 1) * fleet.M).sum())},
        "peaks": {"fp32_tflops": peaks["fp32_flops"] / 1e12, "sm_count": peaks["sm_count"],
                  **{k: v / 1e9 for k, v in peaks.items() if k.endswith("_ops")}, "mufu_unit": "Gop/s"},
    }
    line["e2e"] = run_fleet_e2e(args, fleet, res["shape"], n_steps=min(args.steps, 50))
    stress_in = None
    if not args.no_extras:
        line["plain"] = {"plain_step": run_plain_step(), "one_by_one": run_one_by_one(fleet)}
        line["plain"]["batched_over_one_by_one"] = (value / world) / line["plain"]["one_by_one"]["rollout_steps_per_s"]
        line["closed_loop"] = run_closed_loop(max(args.steps, 100), peaks)
        line["stress"], prob, gpu = run_stress(peaks)
        stress_in = (prob, gpu)
        line["paper_operating_point"] = run_paper_point()
        line["options"] = run_options()
        try:
            line["serving"] = run_serving(args)
        except (ImportError, AttributeError, OSError) as e:
            line["serving"] = {"unavailable": str(e)[:200]}
    clk.stop()
    line["clocks"] = clk.summary()
    line["clocks"]["window"] = (f"every {ClockSampler.LOOP_MS} ms from before the first GPU section to the end "
                                f"of the last")
    line["clocks"]["headline_samples"] = clk.summary(*res["window"])["samples"]
    line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if stress_in and not args.no_oracle:
        line["stress"]["oracle_err"], line["stress"]["cpu_baseline"] = stress_oracle_error(*stress_in)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
