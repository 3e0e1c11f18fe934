"""Python binding of the C ABI in include/mppi.h (libmppi_gb300.so).

Argument marshalling only: every step of the MPPI iteration runs in the
library's CUDA kernels.  PyTorch provides device memory and streams; the
binding passes raw device pointers.  There is no CPU fallback: when the
library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmppi_gb300.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, EAGAIN, ENOTFOUND = 0, -1, -2, -3, -4, -5, -6, -7
N_MAX, M_MAX, K_MAX = 1024, 8192, 1 << 24


class MppiError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else f"{strerror(code)} ({code})")


class Model(C.Structure):
    _fields_ = [("mass", C.c_float), ("g", C.c_float), ("arm_l", C.c_float), ("c_tf", C.c_float),
                ("J", C.c_float * 3), ("T_min", C.c_float), ("T_max", C.c_float), ("motor_clip", C.c_int32),
                ("F_min", C.c_float), ("F_max", C.c_float), ("w_max", C.c_float * 3)]


class Params(C.Structure):
    _fields_ = [("K", C.c_int32), ("N", C.c_int32), ("dt", C.c_float), ("lam", C.c_float),
                ("sigma", C.c_float * 4), ("c_p", C.c_float), ("c_q", C.c_float), ("c_v", C.c_float),
                ("c_w", C.c_float), ("R", C.c_float * 4), ("Rd", C.c_float * 4), ("c_obs", C.c_float),
                ("c_bar", C.c_float), ("beta", C.c_float), ("r_uav", C.c_float), ("quat_metric", C.c_int32),
                ("tail_mode", C.c_int32), ("shift_alpha", C.c_float), ("delay", C.c_float),
                ("seed", C.c_uint64), ("stream_id", C.c_uint32), ("reserved", C.c_int32)]


class Capacity(C.Structure):
    _fields_ = [("max_instances", C.c_int32), ("max_samples", C.c_int64), ("N_max", C.c_int32),
                ("M_max", C.c_int32)]


class Instance(C.Structure):
    _fields_ = [("x_hat", C.c_void_p), ("ref", C.c_void_p), ("obstacles", C.c_void_p), ("u_nom", C.c_void_p),
                ("u_out", C.c_void_p), ("u_cmd", C.c_void_p), ("u_next", C.c_void_p), ("x_next", C.c_void_p),
                ("costs", C.c_void_p), ("status", C.c_void_p), ("iter_dev", C.c_void_p), ("iter", C.c_uint64),
                ("K", C.c_int32), ("N", C.c_int32), ("M", C.c_int32), ("dt", C.c_float), ("lam", C.c_float),
                ("sigma", C.c_float * 4), ("seed", C.c_uint64), ("stream_id", C.c_uint32),
                ("reserved", C.c_int32)]


# The descriptor as a numpy record (same layout), so that a fleet's
# descriptors can be filled with vectorised operations.
INSTANCE_DTYPE = np.dtype(Instance)


class Peaks(C.Structure):
    _fields_ = [("sm_count", C.c_int32), ("reserved", C.c_int32), ("fp32_flops", C.c_double),
                ("fp32_ms", C.c_double), ("ex2_ops", C.c_double), ("lg2_ops", C.c_double),
                ("rsqrt_ops", C.c_double), ("sin_ops", C.c_double), ("cos_ops", C.c_double)]


class Shape(C.Structure):
    _fields_ = [("block", C.c_int32), ("lanes", C.c_int32), ("pipelined", C.c_int32), ("list_margin", C.c_float),
                ("samples_per_thread", C.c_int32)]


class ServerCfg(C.Structure):
    _fields_ = [("max_vehicles", C.c_int32), ("slots", C.c_int32), ("max_batch", C.c_int32), ("N_max", C.c_int32),
                ("M_max", C.c_int32), ("queue_capacity", C.c_int32), ("max_batch_samples", C.c_int64),
                ("hbm_budget_bytes", C.c_int64), ("block", C.c_int32), ("lanes", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("request_id", C.c_uint64), ("vehicle", C.c_int32), ("status", C.c_int32),
                ("u_cmd", C.c_float * 4), ("u0", C.c_float * 4), ("t_submit_us", C.c_double),
                ("t_done_us", C.c_double), ("batch_size", C.c_int32), ("reserved", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("rejected", C.c_int64),
                ("batches", C.c_int64), ("instances", C.c_int64), ("bytes_in_use", C.c_int64),
                ("bytes_budget", C.c_int64), ("busy_us", C.c_double)]


_lib = None
_VP = C.c_void_p
_FP = C.POINTER(C.c_float)


def lib():
    """Loads the library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"MPPI CUDA library not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    L.mppi_version.restype = C.c_char_p
    L.mppi_strerror.restype = C.c_char_p
    L.mppi_strerror.argtypes = [C.c_int]
    L.mppi_create.argtypes = [C.POINTER(Model), C.POINTER(Params), C.POINTER(Capacity), C.POINTER(_VP)]
    L.mppi_destroy.argtypes = [_VP]
    L.mppi_destroy.restype = None
    L.mppi_set_params.argtypes = [_VP, C.POINTER(Params)]
    L.mppi_set_grid.argtypes = [_VP, _VP, C.c_int32, C.c_int32, C.c_int32, _FP, C.c_float]
    L.mppi_set_counters.argtypes = [_VP, _VP]
    L.mppi_set_wait_limit.argtypes = [_VP, C.c_int64, C.c_int32]
    # Pointers passed as addresses (numpy .ctypes.data): the cheapest marshalling.
    L.mppi_solve.argtypes = [_VP, _VP, _VP, _VP, C.c_int32, _VP, C.c_uint64, _VP, _VP, _VP, _VP, _VP]
    L.mppi_solve_async.argtypes = [_VP, _VP, _VP, _VP, C.c_int32, _VP, C.c_uint64, _VP, _VP, _VP, _VP, _VP, _VP,
                                   _VP]
    L.mppi_solve_batch.argtypes = [_VP, C.POINTER(Instance), C.c_int32, _VP]
    L.mppi_solve_batch_graph.argtypes = [_VP, C.POINTER(Instance), C.c_int32, _VP]
    L.mppi_solve_batch_host.argtypes = [_VP, _VP, C.c_int32]
    L.mppi_measure_peaks.argtypes = [C.POINTER(Peaks), _VP]
    L.mppi_sample_noise.argtypes = [C.POINTER(Params), C.c_uint64, C.c_uint32, C.c_int32, C.c_int32, _VP, _VP]
    L.mppi_set_shape.argtypes = [_VP, C.POINTER(Shape)]
    L.mppi_get_shape.argtypes = [_VP, C.c_int32, C.c_int32, C.c_int32, C.POINTER(Shape)]
    L.mppi_autotune.argtypes = [_VP, C.c_int32, C.c_int32, C.c_int32, C.POINTER(Shape), _VP]
    L.mppi_autotune_instance.argtypes = [_VP, C.POINTER(Instance), C.POINTER(Shape), _VP]
    L.mppi_autotune_batch.argtypes = [_VP, C.POINTER(Instance), C.c_int32, C.POINTER(Shape), _VP]
    L.mppi_solve_noalloc.argtypes = [C.POINTER(Model), C.POINTER(Params), _VP, _VP, _VP, C.c_int32, _VP, C.c_uint64,
                                     _VP, _VP, _VP, _VP, _VP, _VP, _VP]
    if hasattr(L, "mppi_server_create"):
        L.mppi_server_create.argtypes = [C.POINTER(Model), C.POINTER(Params), C.POINTER(ServerCfg), C.POINTER(_VP)]
        L.mppi_server_add_vehicle.argtypes = [_VP, C.c_int32, C.c_int32, C.c_float, C.c_float, _FP, _FP, C.c_int32,
                                              _FP, C.c_uint64, C.c_uint32, C.POINTER(C.c_int32)]
        L.mppi_server_remove_vehicle.argtypes = [_VP, C.c_int32]
        L.mppi_server_submit.argtypes = [_VP, C.c_int32, _FP, _FP, C.POINTER(C.c_uint64)]
        L.mppi_server_poll.argtypes = [_VP, C.POINTER(Result), C.c_int32, C.POINTER(C.c_int32)]
        L.mppi_server_drain.argtypes = [_VP, C.c_int32]
        L.mppi_server_export_vehicle.argtypes = [_VP, C.c_int32, _FP, C.POINTER(C.c_uint64)]
        L.mppi_server_import_vehicle.argtypes = [_VP, C.c_int32, _FP, C.c_uint64]
        L.mppi_server_get_stats.argtypes = [_VP, C.POINTER(ServerStats)]
        L.mppi_server_destroy.argtypes = [_VP]
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return lib().mppi_strerror(code).decode()
    except RuntimeError:
        return f"error {code}"


def _check(rc: int, what: str):
    if rc != OK:
        raise MppiError(rc, what)


def make_model(m: dict) -> Model:
    s = Model()
    s.mass, s.g, s.arm_l, s.c_tf = m["mass"], m["g"], m["arm_l"], m["c_tf"]
    s.J[:] = list(m["J"])
    s.T_min, s.T_max, s.motor_clip = m["T_min"], m["T_max"], int(m["motor_clip"])
    s.F_min, s.F_max = m["F_min"], m["F_max"]
    s.w_max[:] = list(m["w_max"])
    return s


def make_params(p: dict) -> Params:
    s = Params()
    s.K, s.N, s.dt, s.lam = int(p["K"]), int(p["N"]), p["dt"], p["lambda"]
    s.sigma[:] = list(p["sigma"])
    s.c_p, s.c_q, s.c_v, s.c_w = p["c_p"], p["c_q"], p["c_v"], p["c_w"]
    s.R[:] = list(p["R"])
    s.Rd[:] = list(p["Rd"])
    s.c_obs, s.c_bar, s.beta, s.r_uav = p["c_obs"], p["c_bar"], p["beta"], p["r_uav"]
    s.quat_metric, s.tail_mode = int(p["quat_metric"]), int(p["tail_mode"])
    s.shift_alpha, s.delay = p["shift_alpha"], p["delay"]
    s.seed, s.stream_id, s.reserved = int(p["seed"]), int(p["stream_id"]), 0
    return s


def _fptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_FP)


def _dptr(t, dtype: str = "float32"):
    """Device address of a torch CUDA tensor, which must be contiguous and of
    the element type the C ABI expects (float32 data, int32 status, int64
    counter); None passes NULL."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous() or str(t.dtype) != "torch." + dtype:
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor, got {t.dtype} on {t.device}"
                         f"{'' if t.is_contiguous() else ' (not contiguous)'}")
    return C.c_void_p(t.data_ptr())


def _sizes(K: int, N: int) -> dict:
    """Element counts the C ABI reads or writes through each buffer."""
    return {"x_hat": 13, "ref": 13 * (N + 1), "u_nom": 4 * N, "u_out": 4 * N, "u_cmd": 4, "u_next": 4 * N,
            "x_next": 13, "costs": K, "status": 1, "iter_dev": 1}


def _check_sizes(K: int, N: int, bufs: dict, minimum=("status", "iter_dev")):
    """Raises ValueError unless every given buffer (numpy array or tensor)
    holds exactly the elements the call uses (at least, for `minimum`), so
    that no call reads or writes past a caller's buffer."""
    want = _sizes(K, N)
    for name, b in bufs.items():
        if b is None:
            continue
        n = b.size if isinstance(b, np.ndarray) else b.numel()
        if n != want[name] and not (name in minimum and n >= want[name]):
            raise ValueError(f"{name}: {n} elements, the step with K={K}, N={N} uses {want[name]}")
    return bufs


def _obstacle_count(obs) -> int:
    if obs is None:
        return 0
    n = obs.size if isinstance(obs, np.ndarray) else obs.numel()
    if n % 4:
        raise ValueError(f"obstacles: {n} elements, not a whole number of (cx, cy, cz, r) rows")
    return n // 4


class _AddressCache:
    """Host addresses of arrays the binding has seen, by identity.

    `ndarray.ctypes.data` costs about a microsecond per call, several times
    per solve.  A closed loop passes the same arrays again (its obstacle
    set) or the arrays a previous solve returned (the next state and
    nominal), whose addresses are known when they are made.  An entry keeps
    its array alive, so its id cannot be reused by another object and its
    data cannot be reallocated (resize refuses a referenced array); the
    cache holds the last few entries only."""

    def __init__(self, size: int = 16):
        self.size = size
        self.d = {}

    def add(self, a, addr: int) -> int:
        d = self.d
        if len(d) >= self.size:
            d.pop(next(iter(d)))
        d[id(a)] = (a, addr)
        return addr

    def get(self, a) -> int:
        e = self.d.get(id(a))
        if e is not None and e[0] is a:
            return e[1]
        return self.add(a, a.ctypes.data)


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Solver:
    """A handle: one vehicle model and one parameter set on the current
    CUDA device, with its own device workspace."""

    def __init__(self, model: dict, params: dict, capacity: dict | None = None):
        self.model, self.params = dict(model), dict(params)
        h = C.c_void_p()
        cap = None
        if capacity is not None:
            cap = Capacity(int(capacity["max_instances"]), int(capacity["max_samples"]), int(capacity["N_max"]),
                           int(capacity["M_max"]))
        self._m, self._p = make_model(model), make_params(params)
        _check(lib().mppi_create(C.byref(self._m), C.byref(self._p), C.byref(cap) if cap else None, C.byref(h)),
               "mppi_create")
        self.h = h
        self._addr = _AddressCache()
        self._blk_t = {}  # ctypes array type per output block size

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().mppi_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params: dict):
        self.params = dict(params)
        self._p = make_params(params)
        _check(lib().mppi_set_params(self.h, C.byref(self._p)), "mppi_set_params")

    def set_grid(self, occ=None, origin=(0.0, 0.0, 0.0), voxel: float = 1.0):
        """mppi_set_grid: occ is a torch uint8 CUDA tensor of shape (nz, ny, nx)
        (kept referenced by the solver), or None to remove the grid."""
        self._grid = occ
        if occ is None:
            _check(lib().mppi_set_grid(self.h, None, 0, 0, 0, None, 0.0), "mppi_set_grid")
            return
        nz, ny, nx = occ.shape
        o = np.ascontiguousarray(origin, np.float32)
        _check(lib().mppi_set_grid(self.h, C.c_void_p(occ.data_ptr()), nx, ny, nz, _fptr(o), float(voxel)),
               "mppi_set_grid")

    def set_counters(self, counters=None):
        """mppi_set_counters: counters is a torch int64 CUDA tensor (>= 1
        element) that later launches add their evaluated obstacle pairs to."""
        self._counters = counters
        _check(lib().mppi_set_counters(self.h, None if counters is None else C.c_void_p(counters.data_ptr())),
               "mppi_set_counters")

    def set_wait_limit(self, polls: int = 0, stall_obstacle_copy: bool = False):
        """mppi_set_wait_limit: bound of the kernel's device-side waits (0:
        default) and the failure-path hook that skips the obstacle copy."""
        _check(lib().mppi_set_wait_limit(self.h, int(polls), 1 if stall_obstacle_copy else 0),
               "mppi_set_wait_limit")

    # ---------------------------------------------------------- host buffers
    def solve(self, x_hat, ref, obstacles, u_nom, it: int, want_costs: bool = False) -> dict:
        """mppi_solve: host numpy in, host numpy out (synchronous)."""
        K, N = int(self.params["K"]), int(self.params["N"])
        x = np.ascontiguousarray(x_hat, np.float32)
        r = np.ascontiguousarray(ref, np.float32)
        o = np.ascontiguousarray(obstacles, np.float32)
        u = np.ascontiguousarray(u_nom, np.float32)
        if x.size != 13 or r.size != 13 * (N + 1) or u.size != 4 * N or o.size % 4:
            _obstacle_count(o)
            _check_sizes(K, N, {"x_hat": x, "ref": r, "u_nom": u})
        o = o.reshape(-1, 4)
        # One allocation for all outputs (each returned array is its own
        # view); a ctypes array gives its address without an ndarray.ctypes
        # object.
        n_out = 8 * N + 17 + (K if want_costs else 0)
        T = self._blk_t.get(n_out)
        if T is None:
            T = self._blk_t[n_out] = C.c_float * n_out
        buf = T()
        base = C.addressof(buf)
        blk = np.frombuffer(buf, np.float32)
        out = {"u_out": blk[:4 * N].reshape(N, 4), "u_cmd": blk[4 * N:4 * N + 4],
               "u_next": blk[4 * N + 4:8 * N + 4].reshape(N, 4), "x_next": blk[8 * N + 4:8 * N + 17],
               "costs": blk[8 * N + 17:] if want_costs else None}
        A = self._addr
        rc = lib().mppi_solve(self.h, A.get(x), A.get(r), A.get(o) if o.size else None, o.shape[0], A.get(u),
                              int(it), base, base + 16 * N, base + 16 * N + 16, base + 32 * N + 16,
                              base + 32 * N + 68 if want_costs else None)
        # The next state and nominal are usually the next call's inputs.
        A.add(out["u_next"], base + 16 * N + 16)
        A.add(out["x_next"], base + 32 * N + 16)
        if rc not in (OK, ENONFINITE):
            raise MppiError(rc, "mppi_solve")
        out["status"] = rc
        return out

    # -------------------------------------------------------- device buffers
    def solve_async(self, x_hat, ref, obstacles, u_nom, it: int, u_out=None, u_cmd=None, u_next=None, x_next=None,
                    costs=None, status=None, stream=None) -> None:
        """mppi_solve_async: torch CUDA tensors in and out, enqueued on stream."""
        M = _obstacle_count(obstacles)
        _check_sizes(int(self.params["K"]), int(self.params["N"]),
                     dict(x_hat=x_hat, ref=ref, u_nom=u_nom, u_out=u_out, u_cmd=u_cmd, u_next=u_next,
                          x_next=x_next, costs=costs, status=status))
        rc = lib().mppi_solve_async(self.h, _dptr(x_hat), _dptr(ref), _dptr(obstacles) if M else None, M,
                                    _dptr(u_nom), int(it), _dptr(u_out), _dptr(u_cmd), _dptr(u_next), _dptr(x_next),
                                    _dptr(costs), _dptr(status, "int32"), _stream_ptr(stream))
        _check(rc, "mppi_solve_async")

    @staticmethod
    def _instances(instances: list):
        arr = (Instance * len(instances))()
        for i, d in enumerate(instances):
            s = arr[i]
            _check_sizes(int(d["K"]), int(d["N"]), {f: d.get(f) for f in _sizes(1, 1)})
            for f in ("x_hat", "ref", "u_nom", "u_out", "u_cmd", "u_next", "x_next", "costs", "status", "iter_dev"):
                t = d.get(f)
                ptr = _dptr(t, "int32" if f == "status" else "int64" if f == "iter_dev" else "float32")
                setattr(s, f, ptr.value if ptr is not None else None)
            obs = d.get("obstacles")
            M = _obstacle_count(obs)
            s.obstacles = _dptr(obs).value if M else None
            s.iter = int(d.get("iter", 0))
            s.K, s.N, s.M = int(d["K"]), int(d["N"]), M
            s.dt, s.lam = float(d["dt"]), float(d["lambda"])
            s.sigma[:] = list(d["sigma"])
            s.seed, s.stream_id, s.reserved = int(d.get("seed", 0)), int(d.get("stream_id", 0)), 0
        return arr

    def solve_batch(self, instances: list, stream=None, graph: bool = False) -> None:
        """mppi_solve_batch(_graph): instances are dicts of torch CUDA tensors
        (x_hat, ref, obstacles, u_nom, and any of u_out, u_cmd, u_next,
        x_next, costs, status, iter_dev) plus K, N, dt, lambda, sigma, seed,
        stream_id, iter; or a record array of INSTANCE_DTYPE holding device
        addresses."""
        if isinstance(instances, np.ndarray):
            # A record array of INSTANCE_DTYPE with device addresses, passed
            # as is (no per-buffer size checks: the caller sized them).
            if instances.dtype != INSTANCE_DTYPE or not instances.flags.c_contiguous:
                raise ValueError("instances must be a contiguous record array of INSTANCE_DTYPE")
            arr, n = C.cast(instances.ctypes.data, C.POINTER(Instance)), instances.size
        else:
            arr, n = self._instances(instances), len(instances)
        fn = lib().mppi_solve_batch_graph if graph else lib().mppi_solve_batch
        _check(fn(self.h, arr, n, _stream_ptr(stream)), "mppi_solve_batch")

    def solve_batch_host(self, instances) -> int:
        """mppi_solve_batch_host: a numpy record array of INSTANCE_DTYPE whose
        pointer fields hold HOST addresses (inputs and outputs), solved
        synchronously; returns the first non-OK instance status (or OK) and
        raises on invalid arguments or a CUDA failure.  The caller keeps the
        addressed arrays alive and sized for each instance's K, N and M."""
        arr = np.ascontiguousarray(instances)
        if arr.dtype != INSTANCE_DTYPE:
            raise ValueError("instances must be a record array of INSTANCE_DTYPE")
        rc = lib().mppi_solve_batch_host(self.h, arr.ctypes.data, arr.size)
        if rc not in (OK, ENONFINITE, ETIMEOUT):
            raise MppiError(rc, "mppi_solve_batch_host")
        return rc

    def autotune_batch(self, instances: list, stream=None):
        """mppi_autotune_batch: the fastest shape for one persistent launch
        of these instances (dicts as for solve_batch; outputs not written)."""
        s = Shape()
        arr = self._instances(instances)
        _check(lib().mppi_autotune_batch(self.h, arr, len(instances), C.byref(s), _stream_ptr(stream)),
               "mppi_autotune_batch")
        return s.block, s.lanes, s.pipelined, s.list_margin, s.samples_per_thread

    def batch_shape(self, instances: list):
        """(block, lanes, pipelined, list_margin, samples_per_thread) a batched launch of these
        instances uses."""
        K = sum(int(d["K"]) for d in instances) // len(instances)
        return self.get_shape(K, max(int(d["N"]) for d in instances),
                              max(_obstacle_count(d.get("obstacles")) for d in instances))

    # ---------------------------------------------------------- launch shape
    def set_shape(self, block: int = 0, lanes: int = 0, pipelined: int = 0, list_margin: float = 0.0,
                  samples_per_thread: int = 1):
        """mppi_set_shape: force a launch shape (all 0: back to the tuned or
        default choice).  list_margin is the obstacle tiling in metres (0:
        default); samples_per_thread 2 packs two samples per thread."""
        s = Shape(block, lanes, pipelined, list_margin, samples_per_thread)
        _check(lib().mppi_set_shape(self.h, C.byref(s)), "mppi_set_shape")

    def get_shape(self, K: int, N: int, M: int):
        """(block, lanes, pipelined, list_margin, samples_per_thread) used for a problem of size (K, N, M)."""
        s = Shape()
        _check(lib().mppi_get_shape(self.h, K, N, M, C.byref(s)), "mppi_get_shape")
        return s.block, s.lanes, s.pipelined, s.list_margin, s.samples_per_thread

    def autotune(self, K: int, N: int, M: int, stream=None):
        """mppi_autotune: the fastest (block, lanes, pipelined, list_margin, samples_per_thread)
        on a synthetic problem of size (K, N, M)."""
        s = Shape()
        _check(lib().mppi_autotune(self.h, K, N, M, C.byref(s), _stream_ptr(stream)), "mppi_autotune")
        return s.block, s.lanes, s.pipelined, s.list_margin, s.samples_per_thread

    def autotune_on(self, instance: dict, stream=None):
        """mppi_autotune_instance: the fastest shape on one of the caller's
        problems (a dict as for solve_batch; its outputs are not written)."""
        s = Shape()
        arr = self._instances([instance])
        _check(lib().mppi_autotune_instance(self.h, arr, C.byref(s), _stream_ptr(stream)), "mppi_autotune_instance")
        return s.block, s.lanes, s.pipelined, s.list_margin, s.samples_per_thread


def solve_noalloc(model: dict, params: dict, x_hat, ref, obstacles, u_nom, it: int, u_out=None, u_cmd=None,
                  u_next=None, x_next=None, costs=None, status=None, stream=None) -> None:
    """mppi_solve_noalloc: the allocation-free step (no handle; scratch in a
    fixed device array; K <= 32768, N <= 256).  torch CUDA tensors in/out."""
    m, p = make_model(model), make_params(params)
    M = _obstacle_count(obstacles)
    _check_sizes(int(params["K"]), int(params["N"]),
                 dict(x_hat=x_hat, ref=ref, u_nom=u_nom, u_out=u_out, u_cmd=u_cmd, u_next=u_next, x_next=x_next,
                      costs=costs, status=status))
    rc = lib().mppi_solve_noalloc(C.byref(m), C.byref(p), _dptr(x_hat), _dptr(ref), _dptr(obstacles) if M else None,
                                  M, _dptr(u_nom), int(it), _dptr(u_out), _dptr(u_cmd), _dptr(u_next),
                                  _dptr(x_next), _dptr(costs), _dptr(status, "int32"), _stream_ptr(stream))
    _check(rc, "mppi_solve_noalloc")


def host_instances(instances: list) -> np.ndarray:
    """A record array of INSTANCE_DTYPE for mppi_solve_batch_host from dicts
    of numpy float32 arrays (x_hat, ref, obstacles, u_nom, and any of u_out,
    u_cmd, u_next, x_next, costs; status an int32 array) plus K, N, dt,
    lambda, sigma, seed, stream_id, iter.  Every array is checked against
    its instance's K and N; the caller keeps the arrays alive."""
    arr = np.zeros(len(instances), INSTANCE_DTYPE)
    for i, d in enumerate(instances):
        K, N = int(d["K"]), int(d["N"])
        _check_sizes(K, N, {f: d.get(f) for f in _sizes(1, 1) if f != "iter_dev"})
        for f in ("x_hat", "ref", "u_nom", "u_out", "u_cmd", "u_next", "x_next", "costs", "status"):
            a = d.get(f)
            if a is None:
                continue
            want = np.int32 if f == "status" else np.float32
            if not isinstance(a, np.ndarray) or a.dtype != want or not a.flags.c_contiguous:
                raise ValueError(f"{f}: expected a contiguous numpy {np.dtype(want).name} array")
            arr[f][i] = a.ctypes.data
        obs = d.get("obstacles")
        M = _obstacle_count(obs)
        if M:
            if obs.dtype != np.float32 or not obs.flags.c_contiguous:
                raise ValueError("obstacles: expected a contiguous numpy float32 array")
            arr["obstacles"][i] = obs.ctypes.data
        arr["iter"][i], arr["K"][i], arr["N"][i], arr["M"][i] = int(d.get("iter", 0)), K, N, M
        arr["dt"][i], arr["lam"][i], arr["sigma"][i] = float(d["dt"]), float(d["lambda"]), list(d["sigma"])
        arr["seed"][i], arr["stream_id"][i] = int(d.get("seed", 0)), int(d.get("stream_id", 0))
    return arr


def measure_peaks(stream=None) -> dict:
    """mppi_measure_peaks: measured FP32 FMA and MUFU throughput of the
    current device."""
    p = Peaks()
    _check(lib().mppi_measure_peaks(C.byref(p), _stream_ptr(stream)), "mppi_measure_peaks")
    return {f: getattr(p, f) for f, _ in Peaks._fields_ if f != "reserved"}


def sample_noise(params: dict, it: int, k0: int, K: int, N: int, out=None, stream=None):
    """mppi_sample_noise: the noise delta u_{k,j} (Sec. III-A) that a solve
    with these parameters at iteration `it` draws, for samples k0 .. k0+K-1
    and steps 0 .. N-1, into `out` (a contiguous CUDA float32 tensor of shape
    (K, N, 4); allocated when None).  Returns `out`."""
    import torch
    if out is None:
        out = torch.empty((K, N, 4), dtype=torch.float32, device="cuda")
    if out.numel() < 4 * K * N:
        raise ValueError("out holds fewer than K*N*4 floats")
    P = make_params(params)
    _check(lib().mppi_sample_noise(C.byref(P), int(it), int(k0), int(K), int(N), _dptr(out), _stream_ptr(stream)),
           "mppi_sample_noise")
    return out


def version() -> str:
    return lib().mppi_version().decode()
