"""ctypes binding of the FP64 CPU oracle (mppi_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests, by the package smoke check and
by the benchmark's CPU-baseline leg.  The product path never imports it.

Every function takes the parameter dictionaries of the shared input module
(model / params) and numpy arrays, converts them to float64 and calls the C
routine of the same name.  See mppi_oracle.c for the equations followed.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mppi_oracle.c")
_LIB = os.environ.get("MPPI_ORACLE_LIB") or os.path.join(_HERE, "liboracle.so")

ENONFINITE = -5


def build(force: bool = False, src: str = _SRC, out: str = None) -> str:
    """Compile the oracle with gcc (-ffp-contract=off so that x86 and Arm
    hosts round identically; OpenMP for the multi-core CPU baseline)."""
    out = out or _LIB
    if os.environ.get("MPPI_ORACLE_LIB") and out == _LIB:
        return _LIB  # a prebuilt library was named explicitly
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-o", tmp, src, "-lm"]
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError:
        cmd.remove("-fopenmp")
        subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(tmp, out)
    return out


class OrcModel(C.Structure):
    _fields_ = [("mass", C.c_double), ("g", C.c_double), ("arm_l", C.c_double), ("c_tf", C.c_double),
                ("J", C.c_double * 3), ("T_min", C.c_double), ("T_max", C.c_double),
                ("motor_clip", C.c_int), ("pad0", C.c_int), ("F_min", C.c_double), ("F_max", C.c_double),
                ("w_max", C.c_double * 3)]


class OrcParams(C.Structure):
    _fields_ = [("K", C.c_int), ("N", C.c_int), ("dt", C.c_double), ("lam", C.c_double),
                ("sigma", C.c_double * 4), ("c_p", C.c_double), ("c_q", C.c_double), ("c_v", C.c_double),
                ("c_w", C.c_double), ("R", C.c_double * 4), ("Rd", C.c_double * 4), ("c_obs", C.c_double),
                ("c_bar", C.c_double), ("beta", C.c_double), ("r_uav", C.c_double),
                ("quat_metric", C.c_int), ("tail_mode", C.c_int), ("shift_alpha", C.c_double),
                ("delay", C.c_double), ("seed", C.c_uint64), ("stream_id", C.c_uint32), ("pad1", C.c_int),
                ("grid", C.c_void_p), ("gx", C.c_int), ("gy", C.c_int), ("gz", C.c_int), ("pad2", C.c_int),
                ("g_origin", C.c_double * 3), ("g_voxel", C.c_double)]


def make_model(m: dict) -> OrcModel:
    s = OrcModel()
    s.mass, s.g, s.arm_l, s.c_tf = m["mass"], m["g"], m["arm_l"], m["c_tf"]
    s.J[:] = list(m["J"])
    s.T_min, s.T_max, s.motor_clip = m["T_min"], m["T_max"], int(m["motor_clip"])
    s.F_min, s.F_max = m["F_min"], m["F_max"]
    s.w_max[:] = list(m["w_max"])
    return s


def make_params(p: dict) -> OrcParams:
    s = OrcParams()
    s.K, s.N, s.dt, s.lam = int(p["K"]), int(p["N"]), p["dt"], p["lambda"]
    s.sigma[:] = list(p["sigma"])
    s.c_p, s.c_q, s.c_v, s.c_w = p["c_p"], p["c_q"], p["c_v"], p["c_w"]
    s.R[:] = list(p["R"])
    s.Rd[:] = list(p["Rd"])
    s.c_obs, s.c_bar, s.beta, s.r_uav = p["c_obs"], p["c_bar"], p["beta"], p["r_uav"]
    s.quat_metric, s.tail_mode = int(p["quat_metric"]), int(p["tail_mode"])
    s.shift_alpha, s.delay = p["shift_alpha"], p["delay"]
    s.seed, s.stream_id = int(p["seed"]), int(p["stream_id"])
    g = p.get("grid")
    if g is not None:
        occ = np.ascontiguousarray(g["occ"], np.uint8)  # shape (gz, gy, gx)
        s._grid_ref = occ  # keep the buffer alive with the struct
        s.grid = occ.ctypes.data
        s.gz, s.gy, s.gx = occ.shape
        s.g_origin[:] = list(g["origin"])
        s.g_voxel = g["voxel"]
    return s


_lib = None
_D = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        MP, PP = C.POINTER(OrcModel), C.POINTER(OrcParams)
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.orc_uniform.restype = C.c_double
        L.orc_uniform.argtypes = [C.c_uint32]
        L.orc_box_muller.argtypes = [C.c_double, C.c_double, _D, _D]
        L.orc_noise.argtypes = [PP, C.c_uint64, C.c_uint32, C.c_uint32, _D]
        L.orc_quat_mul.argtypes = [_D, _D, _D]
        L.orc_rotation_matrix.argtypes = [_D, _D]
        L.orc_dynamics.argtypes = [MP, _D, C.c_double, _D, _D]
        L.orc_rk4_step.argtypes = [MP, _D, C.c_double, _D, C.c_double, _D]
        L.orc_allocation_matrix.argtypes = [MP, _D]
        L.orc_invert4.restype = C.c_int
        L.orc_invert4.argtypes = [_D, _D]
        L.orc_clamp_input.argtypes = [MP, _D, _D]
        L.orc_feasible_input.argtypes = [MP, _D, _D, C.c_double, _D, _D, _D]
        L.orc_quat_distance.restype = C.c_double
        L.orc_quat_distance.argtypes = [_D, _D, C.c_int]
        L.orc_rho_ref.restype = C.c_double
        L.orc_rho_ref.argtypes = [PP, _D, _D]
        L.orc_input_cost.restype = C.c_double
        L.orc_input_cost.argtypes = [PP, _D]
        L.orc_rate_cost.restype = C.c_double
        L.orc_rate_cost.argtypes = [PP, _D, _D]
        L.orc_obstacle_gap.restype = C.c_double
        L.orc_obstacle_gap.argtypes = [PP, _D, _D]
        L.orc_obstacle_cost.restype = C.c_double
        L.orc_obstacle_cost.argtypes = [PP, _D, _D, C.c_int, _D]
        L.orc_rollout.restype = C.c_double
        L.orc_rollout.argtypes = [MP, PP, _D, _D, _D, C.c_int, _D, C.c_uint64, C.c_uint32, _D, _D, _D]
        L.orc_weights.restype = C.c_int
        L.orc_weights.argtypes = [_D, C.c_int, C.c_double, _D]
        L.orc_shift.argtypes = [PP, _D, _D, _D]
        L.orc_mppi_step.restype = C.c_int
        L.orc_mppi_step.argtypes = [MP, PP, _D, _D, _D, C.c_int, _D, C.c_uint64, C.c_int,
                                    _D, _D, _D, _D, _D, _D, _D]
        L.orc_sample_costs.argtypes = [MP, PP, _D, _D, _D, C.c_int, _D, C.c_uint64, C.POINTER(C.c_int),
                                       C.c_int, C.c_int, _D, _D]
        L.orc_noise_block.argtypes = [PP, C.c_uint64, C.c_int, C.c_int, _D]
        L.orc_max_threads.restype = C.c_int
        L.orc_grid_occupied.restype = C.c_int
        L.orc_grid_occupied.argtypes = [PP, _D, _D]
        _lib = L
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D) if a is not None else None


# ---------------------------------------------------------------- primitives

def philox(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def uniform(r: int) -> float:
    return lib().orc_uniform(int(r) & 0xFFFFFFFF)


def box_muller(u0: float, u1: float):
    a, b = C.c_double(), C.c_double()
    lib().orc_box_muller(u0, u1, C.byref(a), C.byref(b))
    return a.value, b.value


def noise(p: dict, it: int, k: int, j: int) -> np.ndarray:
    out = np.zeros(4)
    P = make_params(p)
    lib().orc_noise(C.byref(P), it, k, j, _p(out))
    return out


def noise_block(p: dict, it: int, K: int, N: int) -> np.ndarray:
    out = np.zeros((K, N, 4))
    P = make_params(p)
    lib().orc_noise_block(C.byref(P), it, K, N, _p(out))
    return out


def quat_mul(a, b) -> np.ndarray:
    a, b, o = _d(a), _d(b), np.zeros(4)
    lib().orc_quat_mul(_p(a), _p(b), _p(o))
    return o


def rotation_matrix(q) -> np.ndarray:
    q, o = _d(q), np.zeros(9)
    lib().orc_rotation_matrix(_p(q), _p(o))
    return o.reshape(3, 3)


def dynamics(m: dict, x, F: float, tau) -> np.ndarray:
    x, tau, o = _d(x), _d(tau), np.zeros(13)
    M = make_model(m)
    lib().orc_dynamics(C.byref(M), _p(x), F, _p(tau), _p(o))
    return o


def rk4_step(m: dict, x, F: float, tau, h: float) -> np.ndarray:
    x, tau, o = _d(x), _d(tau), np.zeros(13)
    M = make_model(m)
    lib().orc_rk4_step(C.byref(M), _p(x), F, _p(tau), h, _p(o))
    return o


def allocation_matrix(m: dict) -> np.ndarray:
    o = np.zeros(16)
    M = make_model(m)
    lib().orc_allocation_matrix(C.byref(M), _p(o))
    return o.reshape(4, 4)


def invert4(A) -> np.ndarray:
    A, o = _d(A).reshape(16), np.zeros(16)
    if lib().orc_invert4(_p(A), _p(o)) != 0:
        raise np.linalg.LinAlgError("singular")
    return o.reshape(4, 4)


def clamp_input(m: dict, u) -> np.ndarray:
    u, o = _d(u), np.zeros(4)
    M = make_model(m)
    lib().orc_clamp_input(C.byref(M), _p(u), _p(o))
    return o


def feasible_input(m: dict, x, u_d, dt: float):
    x, u_d = _d(x), _d(u_d)
    F, tau, wc = C.c_double(), np.zeros(3), np.zeros(3)
    M = make_model(m)
    lib().orc_feasible_input(C.byref(M), _p(x), _p(u_d), dt, C.byref(F), _p(tau), _p(wc))
    return F.value, tau, wc


def quat_distance(q1, q2, metric: int = 0) -> float:
    q1, q2 = _d(q1), _d(q2)
    return lib().orc_quat_distance(_p(q1), _p(q2), metric)


def rho_ref(p: dict, x, ref) -> float:
    x, ref = _d(x), _d(ref)
    P = make_params(p)
    return lib().orc_rho_ref(C.byref(P), _p(x), _p(ref))


def input_cost(p: dict, u) -> float:
    u = _d(u)
    P = make_params(p)
    return lib().orc_input_cost(C.byref(P), _p(u))


def rate_cost(p: dict, u_prev, u) -> float:
    a, b = _d(u_prev), _d(u)
    P = make_params(p)
    return lib().orc_rate_cost(C.byref(P), _p(a), _p(b))


def obstacle_gap(p: dict, pos, o) -> float:
    pos, o = _d(pos), _d(o)
    P = make_params(p)
    return lib().orc_obstacle_gap(C.byref(P), _p(pos), _p(o))


def obstacle_cost(p: dict, x, obs) -> float:
    x, obs = _d(x), _d(obs).reshape(-1)
    P = make_params(p)
    g = C.c_double(np.inf)
    return lib().orc_obstacle_cost(C.byref(P), _p(x), _p(obs) if obs.size else None, obs.size // 4, C.byref(g))


def weights(S, lam: float):
    S = _d(S)
    w = np.zeros_like(S)
    rc = lib().orc_weights(_p(S), S.size, lam, _p(w))
    return rc, w


def shift(p: dict, u, u_init) -> np.ndarray:
    u, ui = _d(u), _d(u_init)
    o = np.zeros_like(u)
    P = make_params(p)
    lib().orc_shift(C.byref(P), _p(u), _p(ui), _p(o))
    return o


def rollout(prob: dict, k: int, x0=None, want_traj: bool = False):
    m, p = prob["model"], prob["params"]
    N = int(p["N"])
    x0 = _d(prob["x_hat"] if x0 is None else x0)
    ref, obs, u_nom = _d(prob["ref"]), _d(prob["obstacles"]).reshape(-1), _d(prob["u_nom"])
    traj = np.zeros((N + 1, 13)) if want_traj else None
    useq = np.zeros((N, 4)) if want_traj else None
    g = C.c_double(np.inf)
    M_, P_ = make_model(m), make_params(p)
    S = lib().orc_rollout(C.byref(M_), C.byref(P_), _p(x0), _p(ref), _p(obs) if obs.size else None,
                          obs.size // 4, _p(u_nom), prob["iter"], k, _p(traj), _p(useq), C.byref(g))
    if want_traj:
        return S, traj, useq, g.value
    return S


def mppi_step(prob: dict, n_threads: int = 1) -> dict:
    """One MPPI iteration (Alg. 1 body) in FP64; returns every output."""
    m, p = prob["model"], prob["params"]
    K, N = int(p["K"]), int(p["N"])
    x_hat, ref = _d(prob["x_hat"]), _d(prob["ref"])
    obs, u_nom = _d(prob["obstacles"]).reshape(-1), _d(prob["u_nom"])
    out = {"u_out": np.zeros((N, 4)), "u_cmd": np.zeros(4), "u_next": np.zeros((N, 4)),
           "x_next": np.zeros(13), "costs": np.zeros(K), "weights": np.zeros(K), "min_gap": np.zeros(K)}
    M_, P_ = make_model(m), make_params(p)
    rc = lib().orc_mppi_step(C.byref(M_), C.byref(P_), _p(x_hat), _p(ref), _p(obs) if obs.size else None,
                             obs.size // 4, _p(u_nom), prob["iter"], n_threads,
                             _p(out["u_out"]), _p(out["u_cmd"]), _p(out["u_next"]), _p(out["x_next"]),
                             _p(out["costs"]), _p(out["weights"]), _p(out["min_gap"]))
    out["status"] = rc
    return out


def sample_costs(prob: dict, ks, n_threads: int = 1):
    """S_k for a subset of rollout indices (and their smallest obstacle gap)."""
    m, p = prob["model"], prob["params"]
    ks = np.ascontiguousarray(np.asarray(ks, dtype=np.int32))
    x_hat, ref = _d(prob["x_hat"]), _d(prob["ref"])
    obs, u_nom = _d(prob["obstacles"]).reshape(-1), _d(prob["u_nom"])
    out, gap = np.zeros(ks.size), np.zeros(ks.size)
    M_, P_ = make_model(m), make_params(p)
    lib().orc_sample_costs(C.byref(M_), C.byref(P_), _p(x_hat), _p(ref), _p(obs) if obs.size else None,
                           obs.size // 4, _p(u_nom), prob["iter"], ks.ctypes.data_as(C.POINTER(C.c_int)),
                           ks.size, n_threads, _p(out), _p(gap))
    return out, gap


def grid_occupied(p: dict, pos):
    """(occupied, distance to the nearest occupancy-changing voxel face)."""
    P = make_params(p)
    pos = _d(pos)
    face = C.c_double()
    occ = lib().orc_grid_occupied(C.byref(P), _p(pos), C.byref(face))
    return occ, face.value


def max_threads() -> int:
    return lib().orc_max_threads()
