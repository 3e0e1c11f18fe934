"""Serving: continuous batching of MPPI solves for many vehicles.

Thin binding of the mppi_server_* C ABI plus the fleet load generator used
by the benchmark: every simulated vehicle runs a 100 Hz control clock with
Poisson jitter and submits a solve on each tick unless its previous solve
is still pending (a real-time controller keeps its last command then; the
tick is counted as missed).  Per-vehicle nominal sequences and Philox
counters stay on the device between requests.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np

from . import inputs as I
from . import mppi


def _f(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


class Server:
    def __init__(self, model: dict, params: dict, cfg: dict):
        c = mppi.ServerCfg()
        c.max_vehicles = int(cfg.get("max_vehicles", 1024))
        c.slots = int(cfg.get("slots", 4))
        c.max_batch = int(cfg.get("max_batch", 64))
        c.N_max = int(cfg.get("N_max", 100))
        c.M_max = int(cfg.get("M_max", 64))
        c.queue_capacity = int(cfg.get("queue_capacity", 4096))
        c.max_batch_samples = int(cfg.get("max_batch_samples", 1 << 21))
        c.hbm_budget_bytes = int(cfg.get("hbm_budget_bytes", 8 << 30))
        c.block, c.lanes = int(cfg.get("block", 0)), int(cfg.get("lanes", 0))
        self.cfg = c
        self._m, self._p = mppi.make_model(model), mppi.make_params(params)
        h = C.c_void_p()
        mppi._check(mppi.lib().mppi_server_create(C.byref(self._m), C.byref(self._p), C.byref(c), C.byref(h)),
                    "mppi_server_create")
        self.h = h
        self.N = {}
        self._buf = (mppi.Result * 4096)()

    def add_vehicle(self, K, N, dt, lam, sigma, obstacles, u_init=None, seed=0, stream_id=0) -> int:
        sig = np.ascontiguousarray(sigma, np.float32)
        obs = np.ascontiguousarray(obstacles, np.float32).reshape(-1, 4)
        ui = None if u_init is None else np.ascontiguousarray(u_init, np.float32)
        if sig.size != 4 or (ui is not None and ui.size != 4 * int(N)):
            raise ValueError("sigma needs 4 values and u_init N x 4")
        vid = C.c_int32()
        mppi._check(mppi.lib().mppi_server_add_vehicle(self.h, K, N, dt, lam, _f(sig), _f(obs) if obs.size else None,
                                                       obs.shape[0], _f(ui) if ui is not None else None, seed,
                                                       stream_id, C.byref(vid)), "mppi_server_add_vehicle")
        self.N[vid.value] = N
        return vid.value

    def remove_vehicle(self, vid: int):
        mppi._check(mppi.lib().mppi_server_remove_vehicle(self.h, vid), "mppi_server_remove_vehicle")
        self.N.pop(vid, None)

    def submit(self, vid: int, x_hat: np.ndarray, ref: np.ndarray):
        """Returns the request id, or None when the queue is full.  x_hat
        (13) and ref ((N+1) x 13) are converted to contiguous float32."""
        x = np.ascontiguousarray(x_hat, np.float32)
        r = np.ascontiguousarray(ref, np.float32)
        N = self.N.get(vid)
        if x.size != 13 or (N is not None and r.size != 13 * (N + 1)):
            raise ValueError("x_hat needs 13 values and ref (N+1) x 13 for the vehicle's N")
        rid = C.c_uint64()
        rc = mppi.lib().mppi_server_submit(self.h, vid, _f(x), _f(r), C.byref(rid))
        if rc == mppi.EAGAIN:
            return None
        mppi._check(rc, "mppi_server_submit")
        return rid.value

    def poll(self):
        n = C.c_int32()
        mppi._check(mppi.lib().mppi_server_poll(self.h, self._buf, len(self._buf), C.byref(n)), "mppi_server_poll")
        out = []
        for i in range(n.value):
            r = self._buf[i]
            out.append({"request_id": r.request_id, "vehicle": r.vehicle, "status": r.status,
                        "u_cmd": np.array(r.u_cmd[:], np.float32), "u0": np.array(r.u0[:], np.float32),
                        "latency_us": r.t_done_us - r.t_submit_us, "batch_size": r.batch_size})
        return out

    def drain(self, timeout_ms: int = -1):
        mppi._check(mppi.lib().mppi_server_drain(self.h, timeout_ms), "mppi_server_drain")

    def export_vehicle(self, vid: int):
        u = np.zeros((self.N[vid], 4), np.float32)
        it = C.c_uint64()
        mppi._check(mppi.lib().mppi_server_export_vehicle(self.h, vid, _f(u), C.byref(it)), "export")
        return u, it.value

    def import_vehicle(self, vid: int, u_nom: np.ndarray, it: int):
        u = np.ascontiguousarray(u_nom, np.float32)
        mppi._check(mppi.lib().mppi_server_import_vehicle(self.h, vid, _f(u), it), "import")

    def stats(self) -> dict:
        st = mppi.ServerStats()
        mppi._check(mppi.lib().mppi_server_get_stats(self.h, C.byref(st)), "stats")
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            mppi.lib().mppi_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_fleet(duration_s: float = 5.0, n_vehicles: int = 1000, slots: int = 3, max_batch: int = 512,
              max_batch_samples: int = 1 << 21, warmup_s: float = 1.0, seed: int = 4, rate_hz: float = 100.0,
              queue_capacity: int = 0) -> dict:
    """Serves a fleet (K in {2048, 8192, 32768}, N in {50, 100}, 32 spheres
    each) for `duration_s` after `warmup_s`; reports solves/s,
    rollout-steps/s and p50/p99 latency of the completed requests.  A batch
    takes whatever is queued when a slot frees, up to `max_batch_samples`
    samples (and `max_batch` instances), so its size follows the queue
    depth: small batches at light load, large ones at saturation.  The
    queue holds at most `queue_capacity` requests (0: two full batches per
    slot); submissions beyond it are rejected (backpressure), which bounds
    the queueing delay when the offered load exceeds the GPU."""
    fleet = I.serving_fleet(n_vehicles=n_vehicles, seed=seed)
    mean_K = float(np.mean([v["K"] for v in fleet]))
    queue_capacity = queue_capacity or int(2 * slots * max(1, min(max_batch, max_batch_samples // mean_K)))
    model = I.model(motor_clip=1)
    params = I.params()
    srv = Server(model, params, {"max_vehicles": n_vehicles, "slots": slots, "max_batch": max_batch,
                                 "N_max": 100, "M_max": 32, "queue_capacity": queue_capacity,
                                 "max_batch_samples": max_batch_samples, "hbm_budget_bytes": 64 << 30})
    # A few distinct reference windows shared round-robin (same shapes and
    # magnitudes as per-vehicle windows; the solve cost does not depend on
    # which window a vehicle tracks).
    windows = {}
    for N in (50, 100):
        windows[N] = [I.Trajectory("eight", {"phase": ph}).window(0.0, N, 0.01) for ph in np.linspace(0, 6, 8)]
    vids, xs, refs, work = [], [], [], []
    for i, v in enumerate(fleet):
        vid = srv.add_vehicle(v["K"], v["N"], v["dt"], 1.0, (1.0, 1.0, 1.0, 0.5), v["obstacles"], seed=v["seed"],
                              stream_id=v["stream_id"])
        w = windows[v["N"]][i % 8]
        vids.append(vid)
        refs.append(w)
        xs.append(np.ascontiguousarray(w[0]))
        work.append(v["K"] * v["N"])
    rng = np.random.default_rng(seed)
    n = len(vids)
    next_tick = time.perf_counter() + rng.exponential(1.0 / rate_hz, n)
    pending = np.zeros(n, bool)
    t_start = time.perf_counter()
    t_measure = t_start + warmup_s
    t_end = t_measure + duration_s
    lat, done_steps, done_n, missed, ticks, rejected, bsizes = [], 0, 0, 0, 0, 0, []
    vid_index = {v: i for i, v in enumerate(vids)}
    while True:
        now = time.perf_counter()
        if now >= t_end:
            break
        due = np.nonzero(next_tick <= now)[0]
        for i in due:
            measuring = now >= t_measure
            ticks += measuring
            if pending[i]:
                missed += measuring
            elif srv.submit(vids[i], xs[i], refs[i]) is None:
                rejected += measuring
            else:
                pending[i] = True
            next_tick[i] += rng.exponential(1.0 / rate_hz)
        for r in srv.poll():
            i = vid_index[r["vehicle"]]
            pending[i] = False
            if time.perf_counter() >= t_measure:
                lat.append(r["latency_us"])
                done_steps += work[i]
                done_n += 1
                bsizes.append(r["batch_size"])
        if len(due) == 0:
            time.sleep(0.0002)
    srv.drain(60000)
    st = srv.stats()
    srv.close()
    lat = np.array(lat) if lat else np.array([np.nan])
    return {"workload": f"{n} vehicles at {rate_hz:g} Hz (Poisson), K in {{2048,8192,32768}}, N in {{50,100}}, "
                        f"32 spheres each, {slots} slots, batches of what is queued up to {max_batch_samples} "
                        f"samples",
            "duration_s": duration_s, "solves_per_s": done_n / duration_s,
            "rollout_steps_per_s": done_steps / duration_s,
            "latency_ms": {"p50": float(np.percentile(lat, 50) / 1e3), "p99": float(np.percentile(lat, 99) / 1e3)},
            "offered_per_s": n * rate_hz, "ticks": int(ticks), "missed_ticks": int(missed),
            "rejected": int(rejected), "queue_capacity": queue_capacity,
            "mean_batch": float(np.mean(bsizes)) if bsizes else 0.0,
            "p99_batch": float(np.percentile(bsizes, 99)) if bsizes else 0.0,
            "batches": int(st["batches"]), "dispatcher_host_cores": 1}
