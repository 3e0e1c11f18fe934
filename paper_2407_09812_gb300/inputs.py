"""Seeded synthetic inputs for the MPPI step: vehicle/cost parameters,
initial states, reference windows and obstacle sets.

This module is the one piece shared by the CUDA path's tests/benchmarks and
the CPU oracle.  It holds no arithmetic of the method itself (no dynamics,
cost, noise or weighting): only parameter tables and scenario construction.

Parameter values: Table I (vehicle) and Table II (cost weights) of the paper,
with the workload overrides of the synthetic configurations below (mass
1.0 kg, thrust 0..4g, body rates +-10 rad/s, per-config K, N, dt, lambda,
sigma).  The paper's experiments run on trajectories and obstacle maps from
its simulator; these generators stand in for them with the same shapes and
magnitudes (figure eight with 12 m/s peak speed, a fast sinusoidal line with
12 m/s and 20 m/s^2, spheres and vertical pillars in a bounded box).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

G = 9.81

# Table I of the paper (sim column for limits), mass overridden to 1.0 kg and
# the per-rotor maximum chosen so that 4*T_max equals the 0..4g thrust range.
MODEL_DEFAULT = {
    "mass": 1.0,
    "g": G,
    "arm_l": 0.15,
    "c_tf": 0.012,
    "J": (7.06e-3, 7.06e-3, 13.6e-3),
    "T_min": 0.3,
    "T_max": 1.0 * 4.0 * G / 4.0,
    "motor_clip": 1,
    "F_min": 0.0,
    "F_max": 4.0 * G * 1.0,
    "w_max": (10.0, 10.0, 10.0),
}

# Table II weights; obstacle weights of Sec. IV-D plus the barrier reading.
PARAMS_DEFAULT = {
    "K": 1024,
    "N": 50,
    "dt": 0.02,
    "lambda": 1.0,
    "sigma": (1.0, 1.0, 1.0, 0.5),
    "c_p": 400.0,
    "c_q": 20.0,
    "c_v": 40.0,
    "c_w": 20.0,
    "R": (0.01, 0.05, 0.05, 0.10),
    "Rd": (0.05, 0.10, 0.10, 0.30),
    "c_obs": 1.0e6,
    "c_bar": 100.0,
    "beta": 1.0,
    "r_uav": 0.15,
    "quat_metric": 0,
    "tail_mode": 0,
    "shift_alpha": 1.0,
    "delay": 0.0,
    "seed": 0,
    "stream_id": 0,
}

# Table I as printed: the simulated vehicle and its control limits (Sim
# column).  The collective-thrust box is the four rotors' range.
TABLE_I_VEHICLE = {
    "mass": 1.21,
    "arm_l": 0.15,
    "c_tf": 0.012,
    "J": (7.06e-3, 7.06e-3, 13.6e-3),
    "T_min": 0.3,
    "T_max": 19.0,
    "F_min": 0.0,
    "F_max": 4.0 * 19.0,
    "w_max": (10.0, 10.0, 2.0),
}

# Table II: the controller settings of the paper's experiments.  Sigma is
# printed as a diagonal covariance; the noise generator takes standard
# deviations, so the operating point below passes its square roots.
TABLE_II_MPPI = {
    "dt": 0.1,
    "K": 896,
    "N": 15,
    "lambda": 1.0e-4,
    "Sigma": (0.60, 0.15, 0.15, 0.05),
}


def _f32(v):
    if isinstance(v, (tuple, list)):
        return tuple(float(np.float32(x)) for x in v)
    if isinstance(v, float):
        return float(np.float32(v))
    return v


def f32_exact(d: dict) -> dict:
    """Round every floating value to the nearest float32 so that the FP32
    path and the FP64 oracle see bit-identical parameters."""
    return {k: _f32(v) for k, v in d.items()}


def model(**over) -> dict:
    m = dict(MODEL_DEFAULT)
    m.update(over)
    return f32_exact(m)


def params(**over) -> dict:
    p = dict(PARAMS_DEFAULT)
    p.update(over)
    return f32_exact(p)


def hover_u(m: dict, N: int) -> np.ndarray:
    """u_init of Alg. 1: zero body rates and hover collective thrust."""
    u = np.zeros((N, 4), np.float32)
    u[:, 0] = np.float32(m["mass"] * m["g"])
    return u


def state(p=(0, 0, 0), q=(1, 0, 0, 0), v=(0, 0, 0), w=(0, 0, 0)) -> np.ndarray:
    return np.array(list(p) + list(q) + list(v) + list(w), np.float32)


# --------------------------------------------------------------------------
# Reference trajectories (stand-ins for the paper's simulator trajectories).
# --------------------------------------------------------------------------

def _quat_from_rotation(Rm: np.ndarray) -> np.ndarray:
    """Unit quaternion (w, x, y, z) of a rotation matrix (Shepperd's method)."""
    t = np.trace(Rm)
    if t > 0:
        s = math.sqrt(t + 1.0) * 2
        q = [0.25 * s, (Rm[2, 1] - Rm[1, 2]) / s, (Rm[0, 2] - Rm[2, 0]) / s, (Rm[1, 0] - Rm[0, 1]) / s]
    elif Rm[0, 0] > Rm[1, 1] and Rm[0, 0] > Rm[2, 2]:
        s = math.sqrt(1.0 + Rm[0, 0] - Rm[1, 1] - Rm[2, 2]) * 2
        q = [(Rm[2, 1] - Rm[1, 2]) / s, 0.25 * s, (Rm[0, 1] + Rm[1, 0]) / s, (Rm[0, 2] + Rm[2, 0]) / s]
    elif Rm[1, 1] > Rm[2, 2]:
        s = math.sqrt(1.0 + Rm[1, 1] - Rm[0, 0] - Rm[2, 2]) * 2
        q = [(Rm[0, 2] - Rm[2, 0]) / s, (Rm[0, 1] + Rm[1, 0]) / s, 0.25 * s, (Rm[1, 2] + Rm[2, 1]) / s]
    else:
        s = math.sqrt(1.0 + Rm[2, 2] - Rm[0, 0] - Rm[1, 1]) * 2
        q = [(Rm[1, 0] - Rm[0, 1]) / s, (Rm[0, 2] + Rm[2, 0]) / s, (Rm[1, 2] + Rm[2, 1]) / s, 0.25 * s]
    q = np.array(q)
    q /= np.linalg.norm(q)
    if q[0] < 0:
        q = -q
    return q


def _attitude_for_acceleration(a: np.ndarray, g: float = G) -> np.ndarray:
    """Zero-yaw attitude whose thrust axis points along a - g_vec."""
    zb = a + np.array([0.0, 0.0, g])
    zb = zb / np.linalg.norm(zb)
    xc = np.array([1.0, 0.0, 0.0])
    yb = np.cross(zb, xc)
    yb /= np.linalg.norm(yb)
    xb = np.cross(yb, zb)
    return _quat_from_rotation(np.stack([xb, yb, zb], axis=1))


@dataclass
class Trajectory:
    """Closed-form reference: position/velocity/acceleration of time."""
    kind: str
    params: dict = field(default_factory=dict)

    def pva(self, t: float):
        if self.kind == "hover":
            c = np.array(self.params.get("at", (0.0, 0.0, 0.0)), float)
            return c, np.zeros(3), np.zeros(3)
        if self.kind == "eight":
            # Gerono-style figure eight, 40 m x 20 m, constant phase rate
            # chosen for 12 m/s peak speed.
            A, B, z0 = self.params.get("A", 20.0), self.params.get("B", 10.0), self.params.get("z", 2.5)
            W = self.params.get("omega", 0.4243)
            ph = self.params.get("phase", 0.0)
            s = W * t + ph
            p = np.array([A * math.sin(s), B * math.sin(2 * s), z0])
            v = np.array([A * W * math.cos(s), 2 * B * W * math.cos(2 * s), 0.0])
            a = np.array([-A * W * W * math.sin(s), -4 * B * W * W * math.sin(2 * s), 0.0])
            return p, v, a
        if self.kind == "line":
            # Sinusoidal line: 12 m/s peak speed and 20 m/s^2 peak
            # acceleration (the paper's fastest trajectory, Table III).
            A, W = self.params.get("A", 7.2), self.params.get("omega", 1.6667)
            c = np.array(self.params.get("at", (50.0, 50.0, 5.0)), float)
            d = np.array(self.params.get("dir", (1.0, 0.0, 0.0)), float)
            s = W * t + self.params.get("phase", 0.0)
            return (c + d * A * math.sin(s), d * A * W * math.cos(s), -d * A * W * W * math.sin(s))
        raise ValueError(self.kind)

    def window(self, t0: float, N: int, dt: float) -> np.ndarray:
        """Reference x_ref_0..x_ref_N sampled at t0 + j*dt, shape (N+1, 13)."""
        out = np.zeros((N + 1, 13), np.float64)
        for j in range(N + 1):
            p, v, a = self.pva(t0 + j * dt)
            out[j, 0:3] = p
            out[j, 3:7] = _attitude_for_acceleration(a)
            out[j, 7:10] = v
        return out.astype(np.float32)


# --------------------------------------------------------------------------
# Obstacles: float4 (cx, cy, cz, r); r < 0 marks a vertical cylinder.
# --------------------------------------------------------------------------

def spheres(rng: np.random.Generator, M: int, lo, hi, rmin: float, rmax: float) -> np.ndarray:
    c = rng.uniform(lo, hi, size=(M, 3))
    r = rng.uniform(rmin, rmax, size=(M, 1))
    return np.concatenate([c, r], axis=1).astype(np.float32)


def cylinders(rng: np.random.Generator, M: int, lo, hi, rmin: float, rmax: float) -> np.ndarray:
    o = spheres(rng, M, lo, hi, rmin, rmax)
    o[:, 3] = -o[:, 3]
    return o


# --------------------------------------------------------------------------
# Problems.  A problem is a dict: model, params, x_hat (13,), ref (N+1,13),
# obstacles (M,4), u_nom (N,4), iter (int).  All arrays float32.
# --------------------------------------------------------------------------

def problem(model_d, params_d, x_hat, ref, obstacles, u_nom, it=0) -> dict:
    return {
        "model": model_d,
        "params": params_d,
        "x_hat": np.ascontiguousarray(x_hat, np.float32),
        "ref": np.ascontiguousarray(ref, np.float32),
        "obstacles": np.ascontiguousarray(np.asarray(obstacles, np.float32).reshape(-1, 4)),
        "u_nom": np.ascontiguousarray(u_nom, np.float32),
        "iter": int(it),
    }


def plain_hover(K=1024, N=50, dt=0.02, offset=(0.5, 0.0, 0.0), seed=0, **over) -> dict:
    """Plain single step: hover reference at the origin, start offset
    0.5 m, zero velocity, box-clamped inputs, no obstacles."""
    m = model(motor_clip=0, **{k: v for k, v in over.items() if k in MODEL_DEFAULT})
    p = params(K=K, N=N, dt=dt, seed=seed, **{k: v for k, v in over.items() if k in PARAMS_DEFAULT})
    ref = Trajectory("hover").window(0.0, N, dt)
    return problem(m, p, state(p=offset), ref, np.zeros((0, 4)), hover_u(m, N))


def eight_with_spheres(K=16384, N=100, dt=0.01, M=64, seed=1, t0=0.0, **over) -> dict:
    """Closed-loop tracking step: figure eight, 64 spheres r~U[0.3,1.0] in
    the 40x20x5 m box, per-motor thrust limits."""
    rng = np.random.default_rng(seed)
    m = model(motor_clip=1, **{k: v for k, v in over.items() if k in MODEL_DEFAULT})
    p = params(K=K, N=N, dt=dt, seed=seed, **{k: v for k, v in over.items() if k in PARAMS_DEFAULT})
    traj = Trajectory("eight")
    obs = spheres(rng, M, (-20.0, -10.0, 0.0), (20.0, 10.0, 5.0), 0.3, 1.0)
    ref = traj.window(t0, N, dt)
    x = np.zeros(13, np.float32)
    x[:] = ref[0]
    return problem(m, p, x, ref, obs, hover_u(m, N))


def paper_operating_point(table1_vehicle=False, M=0, seed=1, offset=(0.0, 0.0, 0.0)) -> dict:
    """The paper's own operating point (Table II: K=896, N=15, dt=0.1 s,
    lambda=1e-4, Sigma as a covariance, Table II weights) on the figure
    eight with per-motor limits; the vehicle is the workload default
    (1.0 kg, 0..4g) or, with `table1_vehicle`, Table I's simulated one
    (1.21 kg, rotors 0.3..19 N, yaw rate limit 2 rad/s)."""
    T = TABLE_II_MPPI
    over = {"lambda": T["lambda"], "sigma": tuple(math.sqrt(v) for v in T["Sigma"])}
    if table1_vehicle:
        over.update(TABLE_I_VEHICLE)
    prob = eight_with_spheres(K=T["K"], N=T["N"], dt=T["dt"], M=M, seed=seed, **over)
    prob["x_hat"][0:3] += np.asarray(offset, np.float32)
    return prob


def eight_obstacles_clear_of(traj: "Trajectory", rng, M, t_span, margin=1.2):
    """Spheres of the 40x20x5 box that keep `margin` + r clear of the
    reference path (so that the closed loop is not forced through one)."""
    pts = np.array([traj.pva(t)[0] for t in np.linspace(0, t_span, 2000)])
    out = []
    while len(out) < M:
        o = spheres(rng, 1, (-20.0, -10.0, 0.0), (20.0, 10.0, 5.0), 0.3, 1.0)[0]
        d = np.min(np.linalg.norm(pts - o[:3], axis=1))
        if d > o[3] + margin:
            out.append(o)
    return np.array(out, np.float32).reshape(-1, 4)


def stress_line(K=262144, N=200, dt=0.005, n_spheres=512, n_cyl=512, seed=5, t0=0.0, **over) -> dict:
    """Large-scale stress: sinusoidal line at 12 m/s / 20 m/s^2 through a
    100x100x10 m box of 512 spheres and 512 vertical pillars, r~U[0.2,1.5]."""
    rng = np.random.default_rng(seed)
    m = model(motor_clip=1, **{k: v for k, v in over.items() if k in MODEL_DEFAULT})
    p = params(K=K, N=N, dt=dt, seed=seed, **{k: v for k, v in over.items() if k in PARAMS_DEFAULT})
    obs = np.concatenate([
        spheres(rng, n_spheres, (0.0, 0.0, 0.0), (100.0, 100.0, 10.0), 0.2, 1.5),
        cylinders(rng, n_cyl, (0.0, 0.0, 0.0), (100.0, 100.0, 10.0), 0.2, 1.5),
    ])
    traj = Trajectory("line")
    ref = traj.window(t0, N, dt)
    x = ref[0].copy()
    return problem(m, p, x, ref, obs, hover_u(m, N))


def batched_uneven(n=256, seed=2, dt=0.01, K_range=(1024, 32768), N_range=(30, 150), M_max=128,
                   **over) -> list:
    """Many independent vehicles: K log-uniform in K_range, N uniform in
    N_range, 0..M_max spheres each, random figure-eight phase, initial state
    perturbed around the reference (+-1 m position, N(0, 0.5) m/s velocity)."""
    rng = np.random.default_rng(seed)
    m = model(motor_clip=1, **{k: v for k, v in over.items() if k in MODEL_DEFAULT})
    probs = []
    lo, hi = math.log2(K_range[0]), math.log2(K_range[1])
    for i in range(n):
        K = int(round(2.0 ** rng.uniform(lo, hi)))
        N = int(rng.integers(N_range[0], N_range[1] + 1))
        M = int(rng.integers(0, M_max + 1))
        phase = float(rng.uniform(0, 2 * math.pi))
        p = params(K=K, N=N, dt=dt, seed=seed * 1000003 + i, stream_id=i,
                   **{k: v for k, v in over.items() if k in PARAMS_DEFAULT})
        traj = Trajectory("eight", {"phase": phase})
        ref = traj.window(0.0, N, dt)
        x = ref[0].copy()
        x[0:3] += rng.uniform(-1.0, 1.0, 3).astype(np.float32)
        x[7:10] += rng.normal(0.0, 0.5, 3).astype(np.float32)
        obs = spheres(rng, M, (-20.0, -10.0, 0.0), (20.0, 10.0, 5.0), 0.3, 1.0)
        prob = problem(m, p, x, ref, obs, hover_u(m, N), it=int(rng.integers(0, 1 << 20)))
        prob["phase"] = phase  # the reference's figure-eight phase (for later windows)
        probs.append(prob)
    return probs


def serving_fleet(n_vehicles=1000, seed=4, dt=0.01, Ks=(2048, 8192, 32768), Ns=(50, 100), M=32) -> list:
    """Vehicle specs for the serving loop: K and N drawn uniformly from the
    given sets, M spheres each, random figure-eight phase."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_vehicles):
        K = int(rng.choice(Ks))
        N = int(rng.choice(Ns))
        phase = float(rng.uniform(0, 2 * math.pi))
        obs = spheres(rng, M, (-20.0, -10.0, 0.0), (20.0, 10.0, 5.0), 0.3, 1.0)
        out.append({"K": K, "N": N, "dt": dt, "phase": phase, "obstacles": obs, "seed": seed * 7919 + i,
                    "stream_id": i})
    return out
