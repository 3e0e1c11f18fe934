"""Host logic of the benchmark's fleet (no GPU): every descriptor a
closed-loop step hands to the batched entry points addresses only its own
vehicle's part of the flat buffers, for both ping-pong phases and every
step's reference window, and the host-buffer record builder fills the
descriptors the C ABI reads."""
import numpy as np
import pytest


def test_fleet_descriptors_stay_inside_their_buffers():
    import bench
    from paper_2407_09812_gb300 import mppi
    n_steps = 7
    f = bench.Fleet(n_steps)
    sizes = {"x": f.x0.size, "u": f.u0.size, "ref": f.ref.size, "obs": max(4, f.obs.size), "u_out": f.u0.size,
             "u_cmd": 4 * f.n, "status": f.n}
    base = {"x": [1 << 40, 2 << 40], "u": [3 << 40, 4 << 40], "ref": 5 << 40, "obs": 6 << 40, "u_out": 7 << 40,
            "u_cmd": 8 << 40, "status": 9 << 40}

    def span(ptr, b):  # float offset of ptr in the buffer at b
        d = int(ptr) - b
        assert d % 4 == 0
        return d // 4

    for ping in (0, 1):
        r = f.records(mppi.INSTANCE_DTYPE, base, ping)
        assert r.dtype == mppi.INSTANCE_DTYPE and r.size == f.n
        for step in range(n_steps):
            r["ref"] = base["ref"] + 4 * f.roff + 52 * step
            for i in range(f.n):
                N, M = int(f.N[i]), int(f.M[i])
                for field, buf, length in (("x_hat", base["x"][ping], 13), ("x_next", base["x"][1 - ping], 13),
                                           ("u_nom", base["u"][ping], 4 * N), ("u_next", base["u"][1 - ping], 4 * N),
                                           ("u_out", base["u_out"], 4 * N), ("u_cmd", base["u_cmd"], 4),
                                           ("status", base["status"], 1)):
                    key = {"x_hat": "x", "x_next": "x", "u_nom": "u", "u_next": "u"}.get(field, field)
                    o = span(r[field][i], buf)
                    assert 0 <= o and o + length <= sizes[key], (field, i)
                o = span(r["ref"][i], base["ref"])
                # The window of this step lies inside this vehicle's own trajectory.
                assert f.roff[i] <= o and o + 13 * (N + 1) <= f.roff[i] + f.rlen[i], (i, step)
                if M:
                    o = span(r["obstacles"][i], base["obs"])
                    assert o + 4 * M <= sizes["obs"] and int(r["obstacles"][i]) % 16 == 0
                else:
                    assert int(r["obstacles"][i]) == 0
                assert (int(r["K"][i]), int(r["N"][i]), int(r["M"][i])) == (int(f.K[i]), N, M)
    # The warm start of one phase is the nominal of the other.
    r0, r1 = f.records(mppi.INSTANCE_DTYPE, base, 0), f.records(mppi.INSTANCE_DTYPE, base, 1)
    assert np.array_equal(r0["u_next"], r1["u_nom"]) and np.array_equal(r0["x_next"], r1["x_hat"])
    # Distinct Philox streams per vehicle.
    assert len(set(int(v) for v in r0["stream_id"])) == f.n


def test_host_instance_records_match_the_arrays():
    from paper_2407_09812_gb300 import inputs as I
    from paper_2407_09812_gb300 import mppi
    probs = [I.plain_hover(K=64, N=5), I.eight_with_spheres(K=100, N=7, M=3)]
    dicts = []
    for p in probs:
        K, N = p["params"]["K"], p["params"]["N"]
        dicts.append({"x_hat": p["x_hat"], "ref": p["ref"], "u_nom": p["u_nom"],
                      "obstacles": p["obstacles"] if p["obstacles"].size else None,
                      "u_out": np.zeros((N, 4), np.float32), "status": np.zeros(1, np.int32), "K": K, "N": N,
                      "dt": p["params"]["dt"], "lambda": p["params"]["lambda"], "sigma": p["params"]["sigma"],
                      "seed": 5, "stream_id": 9, "iter": 11})
    r = mppi.host_instances(dicts)
    for d, rec in zip(dicts, r):
        assert rec["x_hat"] == d["x_hat"].ctypes.data and rec["u_out"] == d["u_out"].ctypes.data
        assert rec["u_next"] == 0 and rec["costs"] == 0  # absent outputs are NULL
        assert rec["M"] == (0 if d["obstacles"] is None else d["obstacles"].shape[0])
        assert (rec["K"], rec["N"], rec["iter"], rec["seed"], rec["stream_id"]) == (d["K"], d["N"], 11, 5, 9)
    bad = dict(dicts[0], u_out=np.zeros((5, 4), np.float64))
    with pytest.raises(ValueError):
        mppi.host_instances([bad])
    short = dict(dicts[0], ref=np.zeros((3, 13), np.float32))
    with pytest.raises(ValueError):
        mppi.host_instances([short])


def test_roofline_arithmetic():
    """The roofline entry: algorithmic flop over the launch time against the
    measured FFMA rate, and the MUFU fraction as the time the launch's MUFU
    work needs at the measured rates over the launch time."""
    import bench
    peaks = {"fp32_flops": 80e12, "ex2_ops": 10e12, "lg2_ops": 5e12, "rsqrt_ops": 5e12, "sin_ops": 5e12,
             "cos_ops": 5e12}
    steps, pairs, ms = 1e8, 2e8, 4.0
    flop = steps * bench.FLOP_PER_STEP + pairs * bench.FLOP_PER_PAIR
    r = bench.roofline(flop, bench.mufu_ops(steps, pairs), ms, peaks, 12345, "test")
    assert r["achieved"] == pytest.approx(flop / 4e-3 / 1e12)
    assert r["peak"] == pytest.approx(80.0) and r["frac"] == pytest.approx(r["achieved"] / 80.0)
    mufu_s = (2 * steps + 3 * steps + 2 * steps) / 5e12 + 2 * steps / 5e12 + pairs / 10e12
    assert r["mufu"]["frac"] == pytest.approx(mufu_s / 4e-3)
    assert r["traffic"] == 12345 and r["bound"] == "alu"
    # Traffic is reported only for the kernel source it was captured with.
    assert bench.captured_traffic("no such workload") is None
