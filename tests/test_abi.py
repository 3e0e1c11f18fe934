"""The C-ABI library builds, loads without a GPU, exports every symbol the
public header declares, and validates arguments on the host (no device
work is queued for an invalid call)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2407_09812_gb300 import build as B
    return B.build()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mppi_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("mppi_create", "mppi_solve", "mppi_solve_async", "mppi_solve_batch", "mppi_destroy",
                 "mppi_solve_batch_graph", "mppi_autotune", "mppi_server_create", "mppi_server_submit",
                 "mppi_server_poll", "mppi_solve_noalloc"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    lib = C.CDLL(built)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_validation_rejects_bad_arguments(built):
    from paper_2407_09812_gb300 import inputs as I
    from paper_2407_09812_gb300 import mppi
    L = mppi.lib()
    h = C.c_void_p()
    good_m, good_p = I.model(), I.params()
    cases = [
        (dict(good_m, mass=0.0), good_p),
        (dict(good_m, J=(1e-3, -1.0, 1e-3)), good_p),
        (dict(good_m, T_min=5.0, T_max=1.0), good_p),
        (dict(good_m, motor_clip=2), good_p),
        (good_m, dict(good_p, K=0)),
        (good_m, dict(good_p, N=mppi.N_MAX + 1)),
        (good_m, dict(good_p, dt=0.0)),
        (good_m, dict(good_p, **{"lambda": -1.0})),
        (good_m, dict(good_p, sigma=(1.0, float("nan"), 1.0, 1.0))),
        (good_m, dict(good_p, shift_alpha=0.0)),
        (good_m, dict(good_p, quat_metric=3)),
        (good_m, dict(good_p, c_p=float("inf"))),
    ]
    for m, p in cases:
        mm, pp = mppi.make_model(m), mppi.make_params(p)
        assert L.mppi_create(C.byref(mm), C.byref(pp), None, C.byref(h)) == mppi.EINVAL, (m, p)
        assert not h.value
    assert L.mppi_create(None, None, None, C.byref(h)) == mppi.EINVAL
    assert L.mppi_solve(None, None, None, None, 0, None, 0, None, None, None, None, None) == mppi.EINVAL
    assert L.mppi_solve_batch(None, None, 0, None) == mppi.EINVAL
    assert L.mppi_solve_batch_host(None, None, 0) == mppi.EINVAL
    assert L.mppi_measure_peaks(None, None) == mppi.EINVAL
    assert L.mppi_set_wait_limit(None, 0, 0) == mppi.EINVAL
    assert mppi.strerror(mppi.ENONFINITE) == "every rollout cost was non-finite"


def test_version_string(built):
    from paper_2407_09812_gb300 import mppi
    assert "sm_103a" in mppi.version()


def test_server_host_validation(built):
    """Server configuration errors are caught on the host, before any
    device work: bad sizes (EINVAL) and slot workspaces over the budget
    (ENOMEM)."""
    from paper_2407_09812_gb300 import inputs as I
    from paper_2407_09812_gb300 import mppi
    L = mppi.lib()
    m, p = mppi.make_model(I.model()), mppi.make_params(I.params())
    h = C.c_void_p()

    def cfg(**over):
        c = mppi.ServerCfg()
        vals = dict(max_vehicles=4, slots=2, max_batch=8, N_max=50, M_max=16, queue_capacity=16,
                    max_batch_samples=8192, hbm_budget_bytes=1 << 30, block=0, lanes=0)
        vals.update(over)
        for k, v in vals.items():
            setattr(c, k, v)
        return c

    for bad in (dict(slots=0), dict(max_batch=0), dict(N_max=0), dict(N_max=mppi.N_MAX + 1), dict(M_max=-1),
                dict(queue_capacity=0), dict(block=96, lanes=1), dict(block=128, lanes=3)):
        c = cfg(**bad)
        assert L.mppi_server_create(C.byref(m), C.byref(p), C.byref(c), C.byref(h)) == mppi.EINVAL, bad
    c = cfg(hbm_budget_bytes=1 << 12)
    assert L.mppi_server_create(C.byref(m), C.byref(p), C.byref(c), C.byref(h)) == mppi.ENOMEM
    assert not h.value
    assert L.mppi_server_submit(None, 0, None, None, None) == mppi.EINVAL
    assert L.mppi_server_destroy(None) == mppi.EINVAL


def test_c_client_compiles_and_struct_layouts_match_the_binding(tmp_path):
    """The public header compiles as strict C99 in a C program linked against
    the library, and every public struct has, field by field, the offsets
    and sizes of the Python binding's ctypes mirrors."""
    import subprocess
    from c_client import build_client
    from paper_2407_09812_gb300 import mppi
    exe = build_client(str(tmp_path))
    out = subprocess.run([exe, "layout"], capture_output=True, text=True, check=True).stdout.split("\n")
    mirrors = {"mppi_model": mppi.Model, "mppi_params": mppi.Params, "mppi_capacity": mppi.Capacity,
               "mppi_instance": mppi.Instance, "mppi_shape": mppi.Shape, "mppi_server_cfg": mppi.ServerCfg,
               "mppi_result": mppi.Result, "mppi_server_stats": mppi.ServerStats, "mppi_peaks": mppi.Peaks}
    seen = set()
    for line in filter(None, out):
        struct, field, off, size = line.split()
        py = mirrors[struct]
        if field == "-":
            assert C.sizeof(py) == int(size), (struct, C.sizeof(py), size)
            continue
        f = getattr(py, "lam" if field == "lambda" else field)
        assert (f.offset, f.size) == (int(off), int(size)), (struct, field)
        seen.add((struct, "lam" if field == "lambda" else field))
    for struct, py in mirrors.items():
        assert {(struct, n) for n, _ in py._fields_} <= seen, struct


def test_binding_refuses_buffers_that_do_not_match_the_step(built):
    """The C ABI takes plain pointers and cannot see a buffer's length, so
    the Python binding checks every buffer against K and N before a call:
    a short reference window or a ragged obstacle array never reaches the
    library."""
    import numpy as np
    from paper_2407_09812_gb300 import mppi
    K, N = 64, 7
    good = {"x_hat": np.zeros(13), "ref": np.zeros((N + 1, 13)), "u_nom": np.zeros((N, 4)),
            "u_out": np.zeros((N, 4)), "u_cmd": np.zeros(4), "u_next": np.zeros((N, 4)), "x_next": np.zeros(13),
            "costs": np.zeros(K), "status": np.zeros(1), "iter_dev": np.zeros(1)}
    assert mppi._check_sizes(K, N, good) is good
    for name in good:
        for n in (good[name].size - 1, good[name].size + 1):
            if n < 1 or (name in ("status", "iter_dev") and n > good[name].size):
                continue  # status and the counter may be longer than one element
            with pytest.raises(ValueError, match=name):
                mppi._check_sizes(K, N, dict(good, **{name: np.zeros(n)}))
    assert mppi._obstacle_count(None) == 0 and mppi._obstacle_count(np.zeros((5, 4))) == 5
    with pytest.raises(ValueError):
        mppi._obstacle_count(np.zeros(9))


def test_binding_address_cache_is_by_identity_and_bounded(built):
    """The host-buffer binding remembers the addresses of arrays it has
    seen (or made) by identity; an entry keeps its array alive, so a cached
    id always names the same array, and only the last few are kept."""
    import numpy as np
    from paper_2407_09812_gb300 import mppi
    c = mppi._AddressCache(4)
    a = np.arange(8, dtype=np.float32)
    assert c.get(a) == a.ctypes.data
    v = a[2:]  # a view: its own object, its own address
    assert c.get(v) == a.ctypes.data + 8
    assert c.add(a[1:], a.ctypes.data + 4) == a.ctypes.data + 4
    others = [np.zeros(3, np.float32) for _ in range(6)]
    for o in others:
        assert c.get(o) == o.ctypes.data
    assert len(c.d) <= 4
    assert all(e[0] is not a for e in c.d.values())  # evicted in insertion order
    assert c.get(a) == a.ctypes.data


def test_noalloc_refuses_misaligned_and_oversized_arguments_on_the_host(built):
    """mppi_solve_noalloc checks its arguments before it touches the device:
    a state, reference, nominal or output pointer that is not 4-byte aligned
    (the kernel's scalar accesses would fault), an obstacle pointer that is
    not 16-byte aligned (it is staged by bulk copies), and sizes beyond its
    fixed scratch (K > 32768 or N > 256) all return MPPI_EINVAL.  The
    addresses are never dereferenced, so this runs without a GPU."""
    from paper_2407_09812_gb300 import inputs as I
    from paper_2407_09812_gb300 import mppi
    L = mppi.lib()
    m, p = mppi.make_model(I.model()), mppi.make_params(I.params(K=256, N=10))
    base = 0x7f0000000000  # plausible, 256-byte aligned, never dereferenced
    args = {"x_hat": base, "ref": base + 0x1000, "obstacles": base + 0x2000, "u_nom": base + 0x3000,
            "u_out": base + 0x4000, "u_cmd": base + 0x5000, "u_next": base + 0x6000, "x_next": base + 0x7000,
            "costs": base + 0x8000, "status": base + 0x9000}

    def call(over=None, M=4, pp=p):
        a = dict(args, **(over or {}))
        return L.mppi_solve_noalloc(C.byref(m), C.byref(pp), a["x_hat"], a["ref"], a["obstacles"], M, a["u_nom"],
                                    0, a["u_out"], a["u_cmd"], a["u_next"], a["x_next"], a["costs"], a["status"],
                                    None)

    for name in args:
        off = 8 if name == "obstacles" else 2
        assert call({name: args[name] + off}) == mppi.EINVAL, name
    assert call({"x_hat": None}) == mppi.EINVAL
    assert call({"obstacles": None}) == mppi.EINVAL
    for K, N in ((32769, 10), (256, 257)):
        pp = mppi.make_params(I.params(K=K, N=N))
        assert call(pp=pp) == mppi.EINVAL, (K, N)


def test_sample_noise_refuses_bad_arguments_on_the_host(built):
    """mppi_sample_noise validates before any launch: NULL or misaligned
    output, invalid params, K or N out of range and a sample range past
    2^32 return MPPI_EINVAL (the address is never dereferenced)."""
    from paper_2407_09812_gb300 import inputs as I
    from paper_2407_09812_gb300 import mppi
    L = mppi.lib()
    p = mppi.make_params(I.params(K=256, N=10))
    out = 0x7f0000000000
    assert L.mppi_sample_noise(C.byref(p), 0, 0, 4, 4, None, None) == mppi.EINVAL
    assert L.mppi_sample_noise(None, 0, 0, 4, 4, out, None) == mppi.EINVAL
    assert L.mppi_sample_noise(C.byref(p), 0, 0, 4, 4, out + 4, None) == mppi.EINVAL
    for K, N in ((0, 4), (4, 0), (mppi.K_MAX + 1, 1), (4, mppi.N_MAX + 1)):
        assert L.mppi_sample_noise(C.byref(p), 0, 0, K, N, out, None) == mppi.EINVAL, (K, N)
    assert L.mppi_sample_noise(C.byref(p), 0, (1 << 32) - 3, 4, 1, out, None) == mppi.EINVAL
    bad = mppi.make_params(I.params(sigma=(1.0, float("nan"), 1.0, 1.0)))
    assert L.mppi_sample_noise(C.byref(bad), 0, 0, 4, 4, out, None) == mppi.EINVAL
