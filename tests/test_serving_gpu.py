"""Serving loop (continuous batching, device-resident warm start).

* a vehicle's result is the same served alone and served in a mix of many
  vehicles whose requests arrive while other batches are on the GPU;
* results match the FP64 oracle, and the device-resident nominal and
  Philox counter advance exactly like the host-side warm start;
* admission by device-memory budget and the queue's backpressure.
"""
import numpy as np
import pytest

from parity import U_RTOL, assert_step_close, control_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    assert torch.cuda.is_available()
    from paper_2407_09812_gb300 import build as B
    B.build()
    from paper_2407_09812_gb300 import serve
    return serve


def _fleet(inp, n, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        K = int(rng.choice([300, 1000, 2500]))
        N = int(rng.choice([10, 25, 40]))
        M = int(rng.integers(0, 12))
        ph = float(rng.uniform(0, 6))
        ref = inp.Trajectory("eight", {"phase": ph}).window(0.0, N, 0.01)
        x = ref[0].copy()
        x[0:3] += rng.uniform(-0.5, 0.5, 3).astype(np.float32)
        obs = inp.spheres(rng, M, (-20, -10, 0), (20, 10, 5), 0.3, 1.0)
        p = inp.params(K=K, N=N, dt=0.01, seed=1000 + i, stream_id=i, **{"lambda": [1.0, 80.0][i % 2]})
        out.append(inp.problem(inp.model(motor_clip=1), p, x, ref, obs, inp.hover_u(inp.model(), N), it=0))
    return out


def _server(S, inp, n, slots=3, max_batch=8, shape=(128, 2)):
    return S.Server(inp.model(motor_clip=1), inp.params(),
                    {"max_vehicles": n, "slots": slots, "max_batch": max_batch, "N_max": 40, "M_max": 16,
                     "queue_capacity": 256, "max_batch_samples": 8 * 2500, "hbm_budget_bytes": 2 << 30,
                     "block": shape[0], "lanes": shape[1]})


def _add(srv, p):
    pr = p["params"]
    return srv.add_vehicle(pr["K"], pr["N"], pr["dt"], pr["lambda"], pr["sigma"], p["obstacles"], p["u_nom"],
                           pr["seed"], pr["stream_id"])


def _collect(srv, want):
    got = {}
    import time
    t0 = time.time()
    while len(got) < want and time.time() - t0 < 60:
        for r in srv.poll():
            got[r["request_id"]] = r
    assert len(got) == want
    return got


def test_same_alone_and_in_the_mix_and_matches_oracle(S, orc, inp):
    probs = _fleet(inp, 40)
    target = 7
    # Alone.
    srv = _server(S, inp, 1)
    v = _add(srv, probs[target])
    rid = srv.submit(v, probs[target]["x_hat"], probs[target]["ref"])
    alone = _collect(srv, 1)[rid]
    srv.close()
    # In the mix: 40 vehicles, each submits 3 requests back to back, so
    # later requests arrive while earlier batches run on the 3 slots.
    srv = _server(S, inp, 40)
    vids = [_add(srv, p) for p in probs]
    first = {}
    for rep in range(3):
        for i, p in enumerate(probs):
            rid = srv.submit(vids[i], p["x_hat"], p["ref"])
            if rep == 0:
                first[i] = rid
    res = _collect(srv, 120)
    st = srv.stats()
    srv.close()
    mix = res[first[target]]
    assert alone["status"] == 0 and mix["status"] == 0
    # Same launch shape: bitwise identical; the stated tolerance in any case.
    assert np.array_equal(alone["u_cmd"], mix["u_cmd"]) and np.array_equal(alone["u0"], mix["u0"])
    assert st["batches"] >= 15 and st["completed"] == 120
    assert max(r["batch_size"] for r in res.values()) > 1
    for i in (0, 3, target, 20, 39):
        ref = orc.mppi_step(probs[i], n_threads=8)
        r = res[first[i]]
        sig = probs[i]["params"]["sigma"]
        assert control_err(r["u0"], ref["u_out"][0], sig) <= U_RTOL
        assert control_err(r["u_cmd"], ref["u_cmd"], sig) <= U_RTOL


def test_device_resident_warm_start_advances_like_the_host_loop(S, orc, inp):
    probs = _fleet(inp, 3, seed=9)
    srv = _server(S, inp, 3)
    vids = [_add(srv, p) for p in probs]
    state = [dict(p) for p in probs]
    for step in range(3):
        rids = [srv.submit(v, state[i]["x_hat"], state[i]["ref"]) for i, v in enumerate(vids)]
        res = _collect(srv, 3)
        for i, v in enumerate(vids):
            ref = orc.mppi_step(state[i], n_threads=8)
            r = res[rids[i]]
            sig = state[i]["params"]["sigma"]
            assert control_err(r["u0"], ref["u_out"][0], sig) <= U_RTOL
            u_dev, it = srv.export_vehicle(v)
            assert it == step + 1
            assert control_err(u_dev, ref["u_next"], sig) <= U_RTOL
            state[i] = dict(state[i], u_nom=u_dev, iter=it)
    # Import resets a vehicle (resume from a checkpoint).
    srv.import_vehicle(vids[0], probs[0]["u_nom"], 0)
    rid = srv.submit(vids[0], probs[0]["x_hat"], probs[0]["ref"])
    r = _collect(srv, 1)[rid]
    ref = orc.mppi_step(probs[0], n_threads=8)
    assert control_err(r["u0"], ref["u_out"][0], probs[0]["params"]["sigma"]) <= U_RTOL
    srv.remove_vehicle(vids[2])
    srv.close()


def test_admission_budget_and_backpressure(S, inp):
    from paper_2407_09812_gb300 import mppi
    probs = _fleet(inp, 4, seed=1)
    base = {"max_vehicles": 8, "slots": 1, "max_batch": 2, "N_max": 40, "M_max": 16, "queue_capacity": 3,
            "max_batch_samples": 5000, "block": 128, "lanes": 1}
    # A budget that holds the slot workspace but no vehicle state.
    import paper_2407_09812_gb300.serve as serve_mod
    lo, hi = 1 << 16, 2 << 30
    while hi - lo > 1024:  # smallest budget the server accepts
        mid = (lo + hi) // 2
        try:
            serve_mod.Server(inp.model(), inp.params(), dict(base, hbm_budget_bytes=mid)).close()
            hi = mid
        except mppi.MppiError as e:
            assert e.code == mppi.ENOMEM
            lo = mid
    srv = serve_mod.Server(inp.model(), inp.params(), dict(base, hbm_budget_bytes=hi))
    with pytest.raises(mppi.MppiError) as e:
        _add(srv, probs[0])
    assert e.value.code == mppi.ENOMEM
    srv.close()
    srv = serve_mod.Server(inp.model(), inp.params(), dict(base, hbm_budget_bytes=1 << 30))
    v = _add(srv, probs[0])
    with pytest.raises(ValueError):  # a reference window of the wrong length never reaches the C side
        srv.submit(v, probs[0]["x_hat"], probs[0]["ref"][:-1])
    accepted = [srv.submit(v, probs[0]["x_hat"], probs[0]["ref"]) for _ in range(40)]
    assert any(a is None for a in accepted)  # queue full -> MPPI_EAGAIN
    srv.drain(60000)
    assert srv.stats()["rejected"] >= 1
    srv.close()


def test_remove_vehicle_with_pending_requests(S, orc, inp):
    """Removing a vehicle waits for its queued requests, whose results stay
    available; the vehicle then takes no more requests, a second removal
    finds nothing, a vehicle added in its place starts afresh, and the others are
    unaffected."""
    from paper_2407_09812_gb300 import mppi
    probs = _fleet(inp, 3, seed=21)
    srv = _server(S, inp, 3)
    vids = [_add(srv, p) for p in probs]
    rids = [srv.submit(v, p["x_hat"], p["ref"]) for v, p in zip(vids, probs)]
    srv.remove_vehicle(vids[1])  # returns once its request is done
    with pytest.raises(mppi.MppiError) as e:
        srv.submit(vids[1], probs[1]["x_hat"], probs[1]["ref"])
    assert e.value.code == mppi.ENOTFOUND
    with pytest.raises(mppi.MppiError):
        srv.remove_vehicle(vids[1])
    got = _collect(srv, len(rids))
    assert set(got) == set(rids) and all(got[r]["status"] == 0 for r in rids)
    for i in (0, 1, 2):
        ref = orc.mppi_step(probs[i], n_threads=8)
        assert control_err(got[rids[i]]["u0"], ref["u_out"][0], probs[i]["params"]["sigma"]) <= U_RTOL
    v_new = _add(srv, probs[1])
    r2 = srv.submit(v_new, probs[1]["x_hat"], probs[1]["ref"])
    got2 = _collect(srv, 1)
    assert np.array_equal(got2[r2]["u0"], got[rids[1]]["u0"])  # fresh vehicle: same nominal and counter
    srv.close()


def test_default_shapes_large_batches_match_oracle(S, orc, inp):
    """No forced shape: the server's batched launches take the default shape
    for their total size (up to 8 vehicles of 8192 samples: from two samples
    per thread down to the split pipelined form, by the batch's tile count);
    every result matches the FP64 oracle."""
    rng = np.random.default_rng(11)
    probs = []
    for i in range(12):
        N = 25
        ref = inp.Trajectory("eight", {"phase": float(rng.uniform(0, 6))}).window(0.0, N, 0.01)
        x = ref[0].copy()
        x[0:3] += rng.uniform(-0.5, 0.5, 3).astype(np.float32)
        obs = inp.spheres(rng, 8, (-20, -10, 0), (20, 10, 5), 0.3, 1.0)
        p = inp.params(K=8192, N=N, dt=0.01, seed=500 + i, stream_id=i, **{"lambda": 50.0})
        probs.append(inp.problem(inp.model(motor_clip=1), p, x, ref, obs, inp.hover_u(inp.model(), N), it=0))
    srv = S.Server(inp.model(motor_clip=1), inp.params(),
                   {"max_vehicles": 12, "slots": 2, "max_batch": 8, "N_max": 25, "M_max": 8,
                    "queue_capacity": 64, "max_batch_samples": 8 * 8192, "hbm_budget_bytes": 2 << 30,
                    "block": 0, "lanes": 0})
    vids = [_add(srv, p) for p in probs]
    rids = [srv.submit(v, p["x_hat"], p["ref"]) for v, p in zip(vids, probs)]
    res = _collect(srv, len(rids))
    srv.close()
    assert max(r["batch_size"] for r in res.values()) > 4
    for rid, p in zip(rids, probs):
        r = res[rid]
        assert r["status"] == 0
        ref = orc.mppi_step(p, n_threads=8)
        assert control_err(r["u0"], ref["u_out"][0], p["params"]["sigma"]) <= U_RTOL


def test_serving_fleet_full_size_sampled(S, orc, inp):
    """The benchmark's serving workload at full size: 1000 vehicles (K in
    {2048, 8192, 32768}, N in {50, 100}, 32 spheres each, lambda = 1), the
    benchmark's server configuration (3 slots, batches of up to 2^21 samples
    and 512 vehicles, default launch shapes), one request per vehicle, all
    submitted at once.  Every request completes OK; a fixed sample of the
    vehicles (the first of each (K, N) pair and every 97th) matches a full
    FP64 oracle step: the command, the first updated control, and the
    device-resident warm start and counter."""
    import os
    import time
    fleet = inp.serving_fleet(n_vehicles=1000)
    model, params = inp.model(motor_clip=1), inp.params()
    srv = S.Server(model, params, {"max_vehicles": 1000, "slots": 3, "max_batch": 512, "N_max": 100, "M_max": 32,
                                   "queue_capacity": 1024, "max_batch_samples": 1 << 21,
                                   "hbm_budget_bytes": 64 << 30})
    probs, vids, rids = [], [], []
    for i, v in enumerate(fleet):
        ref = inp.Trajectory("eight", {"phase": v["phase"]}).window(0.0, v["N"], v["dt"])
        p = inp.params(K=v["K"], N=v["N"], dt=v["dt"], seed=v["seed"], stream_id=v["stream_id"],
                       **{"lambda": 1.0, "sigma": (1.0, 1.0, 1.0, 0.5)})
        prob = inp.problem(model, p, np.ascontiguousarray(ref[0]), ref, v["obstacles"], inp.hover_u(model, v["N"]),
                           it=0)
        probs.append(prob)
        vids.append(srv.add_vehicle(v["K"], v["N"], v["dt"], 1.0, (1.0, 1.0, 1.0, 0.5), v["obstacles"],
                                    prob["u_nom"], v["seed"], v["stream_id"]))
    for vid, prob in zip(vids, probs):
        rids.append(srv.submit(vid, prob["x_hat"], prob["ref"]))
    assert all(r is not None for r in rids)
    got, t0 = {}, time.time()
    while len(got) < len(rids) and time.time() - t0 < 120:
        for r in srv.poll():
            got[r["request_id"]] = r
    assert len(got) == len(rids)
    assert all(r["status"] == 0 for r in got.values())
    assert max(r["batch_size"] for r in got.values()) > 1
    first = {}
    for i, v in enumerate(fleet):
        first.setdefault((v["K"], v["N"]), i)
    pick = sorted(set(first.values()) | set(range(0, 1000, 97)))
    for i in pick:
        ref = orc.mppi_step(probs[i], n_threads=os.cpu_count() or 1)
        r = got[rids[i]]
        sig = probs[i]["params"]["sigma"]
        assert control_err(r["u0"], ref["u_out"][0], sig) <= U_RTOL, i
        assert control_err(r["u_cmd"], ref["u_cmd"], sig) <= U_RTOL, i
        u_dev, it = srv.export_vehicle(vids[i])
        assert it == 1
        assert control_err(u_dev, ref["u_next"], sig) <= U_RTOL, i
    srv.close()
