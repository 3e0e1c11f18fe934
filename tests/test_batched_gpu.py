"""Batched persistent launch: many uneven instances in one launch (plain and
replayed from a CUDA graph) give, per instance, the oracle's result within
tolerance and bitwise the same result as solving that instance alone with
the same launch shape."""
import numpy as np
import pytest

from parity import assert_step_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available()
    from paper_2407_09812_gb300 import build as B
    B.build()
    from paper_2407_09812_gb300 import mppi
    return mppi


def _uneven(inp, n=12, seed=7):
    probs = inp.batched_uneven(n=n, seed=seed, K_range=(40, 3000), N_range=(1, 40), M_max=24)
    for i, p in enumerate(probs):
        if i % 3 == 0:
            p["obstacles"] = np.zeros((0, 4), np.float32)
        p["params"] = dict(p["params"], **{"lambda": float([1.0, 50.0, 400.0][i % 3])})
    return probs


def _device(prob, torch):
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    K, N = prob["params"]["K"], prob["params"]["N"]
    d = {"x_hat": t(prob["x_hat"]), "ref": t(prob["ref"]), "u_nom": t(prob["u_nom"]),
         "obstacles": t(prob["obstacles"]) if prob["obstacles"].size else None,
         "u_out": torch.zeros(N, 4, device=dev), "u_cmd": torch.zeros(4, device=dev),
         "u_next": torch.zeros(N, 4, device=dev), "x_next": torch.zeros(13, device=dev),
         "costs": torch.zeros(K, device=dev), "status": torch.zeros(1, dtype=torch.int32, device=dev),
         "K": K, "N": N, "dt": prob["params"]["dt"], "lambda": prob["params"]["lambda"],
         "sigma": prob["params"]["sigma"], "seed": prob["params"]["seed"],
         "stream_id": prob["params"]["stream_id"], "iter": prob["iter"]}
    return d


def _host(d):
    return {k: d[k].cpu().numpy() for k in ("u_out", "u_cmd", "u_next", "x_next", "costs")} | {
        "status": int(d["status"].item())}


def _cap(probs):
    return {"max_instances": len(probs), "max_samples": sum(p["params"]["K"] for p in probs),
            "N_max": max(p["params"]["N"] for p in probs), "M_max": 64}


@pytest.mark.parametrize("graph,shape", [(False, (128, 2, 0)), (True, (128, 2, 0)), (True, (256, 1, 1)),
                                         (True, (128, 1, 0, 0.0, 2)), (False, (512, 1, 3))])
def test_batch_matches_oracle_and_alone(M, orc, inp, graph, shape):
    import torch
    probs = _uneven(inp)
    s = M.Solver(probs[0]["model"], probs[0]["params"], _cap(probs))
    s.set_shape(*shape)
    insts = [_device(p, torch) for p in probs]
    s.solve_batch(insts, graph=graph)
    torch.cuda.synchronize()
    batched = [_host(d) for d in insts]
    # Alone, same launch shape.
    alone_solver = M.Solver(probs[0]["model"], probs[0]["params"], _cap(probs))
    alone_solver.set_shape(*shape)
    for p, b in zip(probs, batched):
        alone_solver.set_params(p["params"])
        d = _device(p, torch)
        alone_solver.solve_async(d["x_hat"], d["ref"], d["obstacles"], d["u_nom"], p["iter"], u_out=d["u_out"],
                                 u_cmd=d["u_cmd"], u_next=d["u_next"], x_next=d["x_next"], costs=d["costs"],
                                 status=d["status"])
        torch.cuda.synchronize()
        a = _host(d)
        for k in ("u_out", "u_cmd", "u_next", "x_next", "costs"):
            assert np.array_equal(a[k], b[k]), (k, p["params"]["K"], p["params"]["N"])
        ref = orc.mppi_step(p, n_threads=8)
        assert b["status"] == 0
        assert_step_close(p, b, ref)
    s.close()
    alone_solver.close()


def test_graph_replay_with_changing_batches(M, orc, inp):
    """One captured graph serves batches of different composition within the
    same capacity bucket; descriptors are updated between replays."""
    import torch
    probs = _uneven(inp, n=10, seed=11)
    s = M.Solver(probs[0]["model"], probs[0]["params"], _cap(probs))
    for subset in (probs[:10], probs[3:7], probs[::2], probs[:10]):
        insts = [_device(p, torch) for p in subset]
        s.solve_batch(insts, graph=True)
        torch.cuda.synchronize()
        for p, d in zip(subset, insts):
            assert_step_close(p, _host(d), orc.mppi_step(p, n_threads=8))
    s.close()


def test_device_counter_and_in_place_warm_start(M, orc, inp):
    """Serving semantics: the nominal lives on the device and is replaced in
    place by the shifted update; the Philox counter is read and advanced on
    the device."""
    import torch
    probs = _uneven(inp, n=4, seed=5)
    s = M.Solver(probs[0]["model"], probs[0]["params"], _cap(probs))
    insts, iters = [], []
    for p in probs:
        d = _device(p, torch)
        it = torch.tensor([p["iter"]], dtype=torch.int64, device="cuda")
        d["iter_dev"] = it
        d["u_next"] = d["u_nom"]  # in place
        insts.append(d)
        iters.append(it)
    expect = [p for p in probs]
    for step in range(3):
        s.solve_batch(insts, graph=True)
        torch.cuda.synchronize()
        for i, (p, d) in enumerate(zip(expect, insts)):
            ref = orc.mppi_step(p, n_threads=8)
            got = _host(d)
            assert_step_close(p, dict(got, u_next=d["u_nom"].cpu().numpy()), ref)
            assert int(iters[i].item()) == p["iter"] + 1
            expect[i] = dict(p, u_nom=d["u_nom"].cpu().numpy(), iter=p["iter"] + 1)
    s.close()


def test_autotuner_picks_a_supported_shape_and_uses_it(M, orc, inp):
    prob = inp.eight_with_spheres(K=3000, N=30, M=48, t0=0.4, **{"lambda": 100.0})
    s = M.Solver(prob["model"], prob["params"])
    before = s.get_shape(3000, 30, 48)
    best = s.autotune(3000, 30, 48)
    if best[2] == 0:  # one thread or 2/4/8/32 lanes per sample
        assert best[0] in (64, 128, 256, 512) and best[1] in (1, 2, 4, 8, 32) and best[0] // best[1] >= 8
    else:  # pipelined: 1-3 dynamics/noise warps plus one or two cost warps per 32 samples
        assert best[2] in (1, 2, 3) and best[1] in (1, 2) and best[0] % (32 * (best[2] + best[1])) == 0
        assert best[0] <= 512
    assert best[3] in (0.25, 0.5, 1.0, 2.0)  # obstacle tiling: kept-list margin [m]
    assert s.get_shape(3000, 30, 48) == best
    assert s.get_shape(3000, 30, 0) == s.get_shape(3000, 30, 0)  # other buckets keep their default
    out = s.solve(prob["x_hat"], prob["ref"], prob["obstacles"], prob["u_nom"], prob["iter"], want_costs=True)
    assert_step_close(prob, out, orc.mppi_step(prob, n_threads=8))
    s.close()
    print("autotune", before, "->", best)


def test_autotune_on_an_instance_leaves_it_untouched(M, orc, inp):
    """Tuning on one of the caller's problems: a supported shape is stored
    for its size bucket, the instance's outputs and device Philox counter
    are not written, and solving with the tuned shape matches the oracle."""
    import torch
    prob = inp.eight_with_spheres(K=4000, N=40, M=64, t0=1.1, **{"lambda": 80.0})
    d = _device(prob, torch)
    sentinel = torch.full_like(d["u_out"], 12345.0)
    d["u_out"].copy_(sentinel)
    d["u_next"] = d["u_nom"]  # in-place warm start would change the nominal if it ran
    it = torch.tensor([prob["iter"]], dtype=torch.int64, device="cuda")
    d["iter_dev"] = it
    nom = d["u_nom"].clone()
    s = M.Solver(prob["model"], prob["params"])
    best = s.autotune_on(d)
    torch.cuda.synchronize()
    assert torch.equal(d["u_out"], sentinel) and torch.equal(d["u_nom"], nom)
    assert int(it.item()) == prob["iter"]
    assert best[3] in (0.25, 0.5, 1.0, 2.0)
    assert s.get_shape(4000, 40, 64) == best
    out = s.solve(prob["x_hat"], prob["ref"], prob["obstacles"], prob["u_nom"], prob["iter"], want_costs=True)
    assert_step_close(prob, out, orc.mppi_step(prob, n_threads=8))
    s.close()
    print("autotune_on", best)


def test_batch_of_one_and_empty_obstacle_sets(M, orc, inp):
    """Degenerate batches: one instance (K = 1 and N = 1 included) and
    instances without obstacles give the alone results and the oracle's."""
    import torch
    probs = [inp.plain_hover(K=1, N=1, seed=9), inp.plain_hover(K=33, N=2, seed=8)]
    for p in probs:
        s = M.Solver(p["model"], p["params"], _cap([p]))
        s.set_shape(128, 1, 0)
        d = _device(p, torch)
        s.solve_batch([d], graph=True)
        torch.cuda.synchronize()
        b = _host(d)
        assert b["status"] == 0
        assert_step_close(p, b, orc.mppi_step(p, n_threads=8))
        a = _device(p, torch)
        s.solve_async(a["x_hat"], a["ref"], None, a["u_nom"], p["iter"], u_out=a["u_out"], u_cmd=a["u_cmd"],
                      u_next=a["u_next"], x_next=a["x_next"], costs=a["costs"], status=a["status"])
        torch.cuda.synchronize()
        for k in ("u_out", "u_cmd", "u_next", "x_next", "costs"):
            assert np.array_equal(_host(a)[k], b[k]), k
        s.close()


def test_host_buffer_batch_matches_device_batch(M, orc, inp):
    """mppi_solve_batch_host (host buffers packed into one pinned block, one
    copy each way, graph-replayed launch) gives bitwise the device-buffer
    batch's results, per instance, and the oracle's; an in-place warm start
    (u_next == u_nom) works on host buffers, and a second call of other
    sizes reuses the packed blocks."""
    import torch
    probs = _uneven(inp, n=9, seed=13)
    s = M.Solver(probs[0]["model"], probs[0]["params"], _cap(probs))
    s.set_shape(128, 1, 0)
    insts = [_device(p, torch) for p in probs]
    s.solve_batch(insts, graph=True)
    torch.cuda.synchronize()
    want = [_host(d) for d in insts]
    host = []
    for p in probs:
        K, N = p["params"]["K"], p["params"]["N"]
        host.append({"x_hat": p["x_hat"].copy(), "ref": p["ref"].copy(), "u_nom": p["u_nom"].copy(),
                     "obstacles": p["obstacles"].copy() if p["obstacles"].size else None,
                     "u_out": np.zeros((N, 4), np.float32), "u_cmd": np.zeros(4, np.float32),
                     "u_next": np.zeros((N, 4), np.float32), "x_next": np.zeros(13, np.float32),
                     "costs": np.zeros(K, np.float32), "status": np.full(1, -99, np.int32), "K": K, "N": N,
                     "dt": p["params"]["dt"], "lambda": p["params"]["lambda"], "sigma": p["params"]["sigma"],
                     "seed": p["params"]["seed"], "stream_id": p["params"]["stream_id"], "iter": p["iter"]})
    assert s.solve_batch_host(M.host_instances(host)) == M.OK
    for p, h, w in zip(probs, host, want):
        assert int(h["status"][0]) == 0
        for k in ("u_out", "u_cmd", "u_next", "x_next", "costs"):
            assert np.array_equal(h[k], w[k]), (k, p["params"]["K"], p["params"]["N"])
        assert_step_close(p, dict(h, status=0), orc.mppi_step(p, n_threads=8))
    # In place, fewer instances, no costs: u_next overwrites the nominal.
    sub = host[2:6]
    for h in sub:
        h["u_next"] = h["u_nom"]
        h["costs"] = None
    nominal = [h["u_nom"].copy() for h in sub]
    assert s.solve_batch_host(M.host_instances(sub)) == M.OK
    for h, w, u0 in zip(sub, want[2:6], nominal):
        assert np.array_equal(h["u_nom"], w["u_next"])
        assert not np.array_equal(h["u_nom"], u0)
    s.close()


def test_batch_autotuner_times_the_batch_and_leaves_it_untouched(M, orc, inp):
    """mppi_autotune_batch times each candidate shape as one persistent
    launch of the caller's batch: it stores a supported shape under the
    batch's key, writes no output and advances no device counter, and the
    tuned batch still matches the oracle."""
    import torch
    probs = _uneven(inp, n=8, seed=17)
    s = M.Solver(probs[0]["model"], probs[0]["params"], _cap(probs))
    insts = [_device(p, torch) for p in probs]
    sentinel = [torch.full_like(d["u_out"], 777.0) for d in insts]
    for d, z in zip(insts, sentinel):
        d["u_out"].copy_(z)
    it = torch.tensor([probs[0]["iter"]], dtype=torch.int64, device="cuda")
    insts[0]["iter_dev"] = it
    best = s.autotune_batch(insts)
    torch.cuda.synchronize()
    assert all(torch.equal(d["u_out"], z) for d, z in zip(insts, sentinel))
    assert int(it.item()) == probs[0]["iter"]
    if best[2] == 0:
        assert best[0] in (64, 128, 256, 512) and best[1] in (1, 2, 4, 8, 32)
    else:
        assert best[2] in (1, 2, 3) and best[1] in (1, 2) and best[0] % (32 * (best[2] + best[1])) == 0
    assert s.batch_shape(insts) == best
    insts[0]["iter_dev"] = None
    s.solve_batch(insts, graph=True)
    torch.cuda.synchronize()
    for p, d in zip(probs, insts):
        assert_step_close(p, _host(d), orc.mppi_step(p, n_threads=8))
    s.close()
    print("autotune_batch", best)


def test_headline_fleet_full_size_sampled(M, orc, inp):
    """The benchmark's headline batch at full size: 256 uneven vehicles (K
    log-uniform in [1024, 32768], N in 30..150, 0..128 spheres, lambda = 1,
    the benchmark's seed), one graph-replayed persistent launch in the shape
    its batch autotuner picks (two samples per thread, block 128, 0.5 m
    margin).  Every instance reports OK with finite outputs; a fixed sample
    of them (the smallest and largest K, N, M and K N, and every 37th) is
    compared with a full FP64 oracle step each, no value taken from the GPU."""
    import os
    import torch
    probs = inp.batched_uneven(n=256, seed=2, dt=0.01)
    cap = {"max_instances": 256, "max_samples": sum(p["params"]["K"] for p in probs), "N_max": 150, "M_max": 128}
    s = M.Solver(probs[0]["model"], probs[0]["params"], cap)
    s.set_shape(128, 1, 0, 0.5, 2)
    insts = [_device(p, torch) for p in probs]
    s.solve_batch(insts, graph=True)
    torch.cuda.synchronize()
    s.close()
    got = [_host(d) for d in insts]
    assert all(g["status"] == 0 for g in got)
    assert all(np.isfinite(g[k]).all() for g in got for k in ("u_out", "u_cmd", "u_next", "x_next", "costs"))
    K = np.array([p["params"]["K"] for p in probs])
    N = np.array([p["params"]["N"] for p in probs])
    Mo = np.array([p["obstacles"].shape[0] for p in probs])
    pick = {int(K.argmin()), int(K.argmax()), int(N.argmin()), int(N.argmax()), int(Mo.argmax()),
            int((K * N).argmax())} | set(range(0, 256, 37))
    for i in sorted(pick):
        ref = orc.mppi_step(probs[i], n_threads=os.cpu_count() or 1)
        assert_step_close(probs[i], got[i], ref)
