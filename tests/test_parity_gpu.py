"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Sizes span several tiles and a ragged tail; the full-size configurations
(closed loop K=16384 N=100 M=64; stress K=262144 N=200 M=1024; the ABI's
limits) are checked on every output against a full FP64 oracle step.
"""
import os

import numpy as np
import pytest

from parity import assert_step_close, control_err, cost_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2407_09812_gb300 import build as B
    B.build()
    from paper_2407_09812_gb300 import mppi
    mppi.lib()
    return mppi


def gpu_solve(M, prob, want_costs=True, shape=None):
    s = M.Solver(prob["model"], prob["params"])
    if shape:
        s.set_shape(*shape)
    out = s.solve(prob["x_hat"], prob["ref"], prob["obstacles"], prob["u_nom"], prob["iter"], want_costs=want_costs)
    s.close()
    return out


def gpu_solve_device(M, prob, shape=None):
    import torch
    dev = torch.device("cuda")
    K, N = prob["params"]["K"], prob["params"]["N"]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    x, r, u = t(prob["x_hat"]), t(prob["ref"]), t(prob["u_nom"])
    o = t(prob["obstacles"]) if prob["obstacles"].size else None
    out = {k: torch.zeros(n, dtype=torch.float32, device=dev) for k, n in
           (("u_out", (N, 4)), ("u_cmd", 4), ("u_next", (N, 4)), ("x_next", 13), ("costs", K))}
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    s = M.Solver(prob["model"], prob["params"])
    if shape:
        s.set_shape(*shape)
    s.solve_async(x, r, o, u, prob["iter"], status=status, **out)
    torch.cuda.synchronize()
    s.close()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["status"] = int(status.item())
    return res


def test_plain_hover_full_size(M, orc, inp):
    prob = inp.plain_hover()  # K=1024, N=50, dt=0.02, box clamp
    ref = orc.mppi_step(prob, n_threads=8)
    g = gpu_solve(M, prob)
    e = assert_step_close(prob, g, ref)
    d = gpu_solve_device(M, prob)
    assert_step_close(prob, d, ref)
    for k in ("u_out", "u_next", "u_cmd", "x_next", "costs"):
        assert np.array_equal(g[k], d[k]), k  # host and device entry points agree bitwise
    print("plain hover errors", e)


@pytest.mark.parametrize("tiles", ["32S", "32S+1", "128S+1", "256S+1", "512S"])
def test_default_shape_regimes_match_oracle(M, orc, inp, tiles):
    """Untuned sizes in each regime of the default launch shape on this GPU's
    S SMs (split pipelined form with 32- and 64-sample tiles, two-warp
    pipelined form, one thread per sample, two samples per thread), ragged
    where the regime allows, through the host-buffer entry point, against
    the full FP64 oracle step."""
    import torch
    S = torch.cuda.get_device_properties(0).multi_processor_count
    K = {"32S": 32 * S, "32S+1": 32 * S + 1, "128S+1": 128 * S + 1, "256S+1": 256 * S + 1, "512S": 512 * S}[tiles]
    prob = inp.eight_with_spheres(K=K, N=9, M=24, t0=0.6, **{"lambda": 150.0})
    want = {"32S": (128, 1, 3, 1), "32S+1": (256, 1, 3, 1), "128S+1": (256, 1, 1, 1), "256S+1": (128, 1, 0, 1),
            "512S": (128, 1, 0, 2)}[tiles]
    s = M.Solver(prob["model"], prob["params"])
    got = s.get_shape(K, 9, 24)
    s.close()
    assert got[:3] + got[4:] == want, got
    assert_step_close(prob, gpu_solve(M, prob), orc.mppi_step(prob, n_threads=os.cpu_count() or 1))


@pytest.mark.parametrize("K,N", [(1, 1), (7, 3), (129, 5), (1000, 17), (4097, 2), (300, 130)])
def test_ragged_sizes(M, orc, inp, K, N):
    prob = inp.plain_hover(K=K, N=N, dt=0.02, seed=K * 31 + N)
    ref = orc.mppi_step(prob, n_threads=8)
    assert_step_close(prob, gpu_solve(M, prob), ref)


@pytest.mark.parametrize("lam", [1.0, 300.0, 3000.0])
def test_obstacles_and_motor_limits(M, orc, inp, lam):
    prob = inp.eight_with_spheres(K=2048, N=40, M=64, t0=1.3, **{"lambda": lam})
    rng = np.random.default_rng(9)
    pillars = inp.cylinders(rng, 16, (-20.0, -10.0, 0.0), (20.0, 10.0, 5.0), 0.3, 1.0)
    prob["obstacles"] = np.ascontiguousarray(np.concatenate([prob["obstacles"], pillars]))
    ref = orc.mppi_step(prob, n_threads=8)
    e = assert_step_close(prob, gpu_solve(M, prob), ref)
    print("obstacles lambda", lam, e, "ess", 1.0 / np.sum(ref["weights"] ** 2))


def test_collisions_in_rollouts(M, orc, inp):
    # Obstacles placed on the reference path so that many rollouts collide.
    prob = inp.eight_with_spheres(K=1024, N=30, M=8, t0=0.0)
    ref_path = prob["ref"][::4, 0:3]
    obs = np.concatenate([ref_path[:8], np.full((8, 1), 0.5, np.float32)], axis=1).astype(np.float32)
    obs[:, 1] += 0.7
    prob["obstacles"] = np.ascontiguousarray(obs)
    ref = orc.mppi_step(prob, n_threads=8)
    assert np.mean(ref["costs"] >= prob["params"]["c_obs"]) > 0.05  # many rollouts collide
    assert_step_close(prob, gpu_solve(M, prob), ref)


def test_temperature_limits_and_zero_noise(M, orc, inp):
    base = inp.eight_with_spheres(K=777, N=12, M=16, t0=2.0)
    for over in ({"lambda": 1e-30}, {"lambda": 1e30}, {"sigma": (0.0, 0.0, 0.0, 0.0)}, {"K": 1}):
        prob = dict(base, params=dict(base["params"], **over))
        ref = orc.mppi_step(prob, n_threads=8)
        g = gpu_solve(M, prob)
        assert_step_close(prob, g, ref)
        if "sigma" in over:
            assert np.array_equal(g["u_out"], prob["u_nom"])


@pytest.mark.parametrize("shape", [None, (128, 1, 0, 0.0, 2), (512, 1, 3)])
@pytest.mark.parametrize("over", [{"quat_metric": 1}, {"tail_mode": 1}, {"shift_alpha": 0.25},
                                  {"delay": 0.004}, {"lambda": 20.0, "shift_alpha": 0.1, "tail_mode": 1}])
def test_step_options(M, orc, inp, over, shape):
    base = inp.eight_with_spheres(K=1500, N=25, M=20, t0=0.7)
    prob = dict(base, params=dict(base["params"], **over))
    ref = orc.mppi_step(prob, n_threads=8)
    assert_step_close(prob, gpu_solve(M, prob, shape=shape), ref)


def test_nonfinite_state_reports_and_keeps_nominal(M, inp):
    prob = inp.plain_hover(K=256, N=10)
    prob["x_hat"] = prob["x_hat"].copy()
    prob["x_hat"][8] = np.nan
    g = gpu_solve(M, prob)
    assert g["status"] == M.ENONFINITE
    assert np.array_equal(g["u_out"], prob["u_nom"])


def test_every_launch_shape_matches_and_is_deterministic(M, orc, inp):
    prob = inp.eight_with_spheres(K=3000, N=20, M=40, t0=3.0, **{"lambda": 500.0})
    ref = orc.mppi_step(prob, n_threads=8)
    shapes = [(b, l, 0, 0.0) for b in (64, 128, 256, 512) for l in (1, 2, 4, 8)]
    shapes += [(64, 32, 0, 0.0), (256, 32, 0, 0.0), (512, 32, 0, 0.0)]
    shapes += [(128, 1, 1, 0.0), (256, 1, 1, 0.0), (512, 1, 1, 0.0), (96, 2, 1, 0.0), (192, 2, 1, 0.0),
               (384, 2, 1, 0.0)]
    shapes += [(96, 1, 2, 0.0), (192, 1, 2, 0.0), (384, 1, 2, 0.0), (256, 2, 2, 0.0), (512, 2, 2, 0.0)]
    shapes += [(128, 1, 3, 0.0), (256, 1, 3, 0.0), (512, 1, 3, 0.0), (160, 2, 3, 0.0), (480, 2, 3, 0.0)]
    shapes += [(64, 1, 0, 0.0, 2), (128, 1, 0, 0.0, 2), (128, 1, 0, 3.0, 2)]
    shapes += [(128, 1, 0, 0.25), (128, 4, 0, 3.0), (256, 1, 1, 2.0), (256, 32, 0, 0.5)]
    for shape in shapes:
        a = gpu_solve(M, prob, shape=shape)
        assert_step_close(prob, a, ref)
        b = gpu_solve(M, prob, shape=shape)
        for k in ("u_out", "costs", "u_cmd"):
            assert np.array_equal(a[k], b[k]), (shape, k)


@pytest.mark.parametrize("K,N,Mo", [(16384, 100, 64), (1000, 1, 3), (257, 7, 0), (3000, 37, 40)])
def test_pipelined_form_matches_one_thread_per_sample(M, orc, inp, K, N, Mo):
    """The pipelined form (dynamics and cost threads per sample, handing
    states over through mbarrier-guarded rings; with a noise thread too)
    gives the per-sample costs of one thread per sample to FP32 rounding
    (the same arithmetic compiled in two places) and matches the oracle."""
    prob = inp.eight_with_spheres(K=K, N=N, M=Mo, t0=0.6, **{"lambda": 200.0})
    if Mo == 0:
        prob["obstacles"] = np.zeros((0, 4), np.float32)
    b = gpu_solve(M, prob, shape=(128, 1, 0))
    ref = orc.mppi_step(prob, n_threads=16)
    for shape in ((256, 1, 1), (384, 2, 1), (384, 1, 2), (512, 2, 2), (512, 1, 3), (320, 2, 3)):
        a = gpu_solve(M, prob, shape=shape)
        assert cost_err(a["costs"], b["costs"])[0] <= 1e-6
        assert_step_close(prob, a, ref)
    # The noise thread's form (pipelined = 2) draws the same noise and runs
    # the same dynamics arithmetic: with the same samples per block its
    # per-sample costs are bitwise the two-warp form's.  The update is equal
    # to rounding: the tile's weighted noise sum splits each step's
    # contributors over (threads per block / N) groups, 384 threads here
    # against 256.
    two, three = gpu_solve(M, prob, shape=(256, 1, 1)), gpu_solve(M, prob, shape=(384, 1, 2))
    assert np.array_equal(two["costs"], three["costs"])
    sig = prob["params"]["sigma"]
    for k in ("u_out", "u_next", "u_cmd"):
        assert control_err(three[k], two[k], sig) <= 1e-6, k
    # The split form (pipelined = 3: attitude and translation threads, the
    # noise thread forming the clamped control) runs the same operations on
    # other threads: per-sample costs bitwise those of the forms above.
    four = gpu_solve(M, prob, shape=(512, 1, 3))
    assert np.array_equal(four["costs"], two["costs"])
    for k in ("u_out", "u_next", "u_cmd"):
        assert control_err(four[k], two[k], sig) <= 1e-6, k


@pytest.mark.parametrize("K,N,Mo", [(16384, 100, 64), (3001, 37, 40), (129, 5, 0), (1000, 1, 3)])
def test_two_samples_per_thread_match_one(M, orc, inp, K, N, Mo):
    """Two samples per thread run each sample's operations as one sample per
    thread, packed across the two; the assembler fuses some packed
    multiply-add pairs that the one-sample code rounds separately, so the
    per-sample costs agree to FP32 rounding (measured: a few ulp), the update
    too (the tiles also hold twice the samples, so the merge groups the
    weighted sums differently), and both match the oracle; ragged tails
    included."""
    prob = inp.eight_with_spheres(K=K, N=N, M=max(Mo, 1), t0=0.9, **{"lambda": 150.0})
    if Mo == 0:
        prob["obstacles"] = np.zeros((0, 4), np.float32)
    one = gpu_solve(M, prob, shape=(128, 1, 0))
    sig = prob["params"]["sigma"]
    for shape in ((64, 1, 0, 0.0, 2), (128, 1, 0, 0.0, 2)):
        two = gpu_solve(M, prob, shape=shape)
        assert cost_err(two["costs"], one["costs"])[0] <= 2e-6, shape
        for k in ("u_out", "u_next", "u_cmd"):
            assert control_err(two[k], one[k], sig) <= 1e-6, (shape, k)
    if K * N <= 200000:
        assert_step_close(prob, one, orc.mppi_step(prob, n_threads=16))


def test_closed_loop_full_size(M, orc, inp):
    """K=16384, N=100, dt=0.01, 64 spheres, figure eight: five closed-loop
    steps; at every step the oracle is fed the GPU's state and nominal."""
    prob = inp.eight_with_spheres()
    s = M.Solver(prob["model"], prob["params"])
    x, u = prob["x_hat"].copy(), prob["u_nom"].copy()
    traj = inp.Trajectory("eight")
    worst = {}
    for t in range(5):
        step = dict(prob, x_hat=x, u_nom=u, ref=traj.window(0.01 * t, 100, 0.01), iter=t)
        g = s.solve(step["x_hat"], step["ref"], step["obstacles"], step["u_nom"], t, want_costs=True)
        ref = orc.mppi_step(step, n_threads=16)
        e = assert_step_close(step, g, ref)
        worst = {k: max(worst.get(k, 0), v) for k, v in e.items()}
        x, u = g["x_next"], g["u_next"]
    s.close()
    print("closed loop worst", worst)


def test_stress_full_size(M, orc, inp):
    """K=262144, N=200, dt=0.005, 512 spheres + 512 pillars: every
    per-sample cost, the updated nominal, the warm start and the command
    against one full FP64 oracle step on all host cores (Eq. cost_2,
    Eq. u_update); the GPU's x_next against the oracle's is reported."""
    prob = inp.stress_line()
    g = gpu_solve(M, prob)
    ref = orc.mppi_step(prob, n_threads=os.cpu_count() or 1)
    e = assert_step_close(prob, g, ref)
    print("stress errors", e, "ess", 1.0 / np.sum(ref["weights"] ** 2))


def test_maximum_sizes(M, orc, inp):
    """The ABI's limits, each at the largest value with the others small,
    against the full FP64 oracle step: N = N_MAX steps, M = M_MAX
    obstacles, and K = K_MAX samples (every one of the 2^24 costs and the
    update)."""
    prob = inp.eight_with_spheres(K=300, N=M.N_MAX, dt=0.002, M=16, t0=0.3, **{"lambda": 100.0})
    assert_step_close(prob, gpu_solve(M, prob), orc.mppi_step(prob, n_threads=16))
    prob = inp.eight_with_spheres(K=256, N=8, M=M.M_MAX, t0=0.3, **{"lambda": 100.0})
    g = gpu_solve(M, prob)
    assert g["status"] == M.OK
    assert_step_close(prob, g, orc.mppi_step(prob, n_threads=16))
    prob = inp.plain_hover(K=M.K_MAX, N=1, seed=3)
    g = gpu_solve(M, prob)
    ref = orc.mppi_step(prob, n_threads=os.cpu_count() or 1)
    e = assert_step_close(prob, g, ref)
    print("K_MAX errors", e, "ess", 1.0 / np.sum(ref["weights"] ** 2))


@pytest.mark.parametrize("shape", [None, (128, 1, 0, 0.0, 2), (512, 1, 3)])
def test_grid_collision_module(M, orc, inp, shape):
    """Occupancy voxel grid as the collision module (with spheres too):
    the GPU's per-state lookup and indicator match the oracle (one thread
    per sample, two samples per thread, the split pipelined form)."""
    import torch
    prob = inp.eight_with_spheres(K=2048, N=40, M=16, t0=0.9, **{"lambda": 300.0})
    rng = np.random.default_rng(21)
    occ = (rng.uniform(size=(12, 44, 84)) < 0.02).astype(np.uint8)  # (z, y, x), 0.5 m voxels
    origin, voxel = (-21.0, -11.0, -0.5), 0.5
    # A wall of occupied voxels across the path ahead, so many rollouts hit it.
    wx, wy, wz = ((prob["ref"][30, :3] - np.array(origin)) / voxel).astype(int)
    occ[wz - 1:wz + 1, wy - 1:wy + 1, wx:wx + 1] = 1
    prob["params"] = dict(prob["params"], grid={"occ": occ, "origin": origin, "voxel": voxel})
    ref = orc.mppi_step(prob, n_threads=8)
    assert np.mean(ref["costs"] >= prob["params"]["c_obs"]) > 0.05  # the grid is hit by many rollouts
    s = M.Solver(prob["model"], prob["params"])
    if shape:
        s.set_shape(*shape)
    s.set_grid(torch.from_numpy(occ).cuda(), origin, voxel)
    g = s.solve(prob["x_hat"], prob["ref"], prob["obstacles"], prob["u_nom"], prob["iter"], want_costs=True)
    e = assert_step_close(prob, g, ref)
    s.set_grid(None)
    g2 = s.solve(prob["x_hat"], prob["ref"], prob["obstacles"], prob["u_nom"], prob["iter"], want_costs=True)
    assert np.mean(g2["costs"] < g["costs"]) > 0.05  # removing the grid removes its penalties
    s.close()
    print("grid module errors", e)


@pytest.mark.parametrize("shape", [None, (128, 1, 0, 0.0, 2)])
def test_evaluated_pair_counter(M, orc, inp, shape):
    """The measurement hook counts evaluated (state, obstacle) pairs: all of
    them when nothing can be culled (beta = 0: the barrier never vanishes),
    fewer with the default barrier; the results stay within tolerance (ragged
    last tile included)."""
    import torch
    prob = inp.eight_with_spheres(K=1000, N=20, M=40, t0=0.2)
    for beta, exact in ((0.0, True), (1.0, False)):
        p = dict(prob, params=dict(prob["params"], beta=beta))
        s = M.Solver(p["model"], p["params"])
        if shape:
            s.set_shape(*shape)
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        s.set_counters(cnt)
        g = s.solve(p["x_hat"], p["ref"], p["obstacles"], p["u_nom"], p["iter"], want_costs=True)
        s.close()
        total = 1000 * 21 * 40
        n = int(cnt.item())
        if exact:
            assert n == total
        else:
            assert 0 < n < total
        assert_step_close(p, g, orc.mppi_step(p, n_threads=8))


@pytest.mark.parametrize("shape", [(128, 1, 0), (256, 1, 1), (128, 2, 0), (384, 2, 1), (128, 1, 0, 0.25),
                                   (256, 1, 1, 3.0), (256, 32, 0), (128, 1, 0, 0.5, 2), (512, 1, 3, 1.0)])
def test_reused_kept_lists_equal_per_step_culling(M, inp, shape):
    """A warp's kept-obstacle list is built for its box grown by a margin and
    reused while its positions stay inside; launches that count evaluated
    pairs cull every step with the unexpanded box instead.  The obstacles
    kept only by the margin add exactly +0, so with one lane per sample the
    per-sample costs and the update are bitwise those of per-step culling
    (with several lanes the lanes' shares are grouped differently: equal to
    rounding).  Cases: 64 spheres; 1024 spheres and cylinders (lists that
    overflow their 64 entries fall back to chunked scoring)."""
    import torch
    probs = [inp.eight_with_spheres(K=3000, N=60, M=64, t0=0.7),
             inp.stress_line(K=2048, N=80)]
    for prob in probs:
        outs = []
        for counting in (False, True):
            s = M.Solver(prob["model"], prob["params"])
            s.set_shape(*shape)
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            if counting:
                s.set_counters(cnt)
            outs.append(s.solve(prob["x_hat"], prob["ref"], prob["obstacles"], prob["u_nom"], prob["iter"],
                                want_costs=True))
            s.close()
        reuse, per_step = outs
        if shape[1] == 1:
            for k in ("costs", "u_out", "u_next", "u_cmd", "x_next"):
                assert np.array_equal(reuse[k], per_step[k]), (k, prob["params"]["K"])
        else:
            c0, c1 = reuse["costs"].astype(np.float64), per_step["costs"].astype(np.float64)
            assert np.max(np.abs(c0 - c1) / np.maximum(np.abs(c1), 1.0)) <= 1e-6


@pytest.mark.parametrize("table1_vehicle", [False, True])
def test_paper_operating_point(M, orc, inp, table1_vehicle):
    """Table II: K=896, N=15, dt=0.1 s, lambda=1e-4, Sigma=diag(0.60, 0.15,
    0.15, 0.05) as a covariance, Table II weights, motor limits; on the
    workload vehicle and on Table I's simulated one (1.21 kg, rotors
    0.3..19 N, yaw rate limit 2 rad/s)."""
    prob = inp.paper_operating_point(table1_vehicle=table1_vehicle, offset=(0.3, -0.2, 0.1))
    for it in range(3):
        p = dict(prob, iter=it)
        assert_step_close(p, gpu_solve(M, p), orc.mppi_step(p, n_threads=8))


@pytest.mark.parametrize("log2_term", [-20.0, -40.0, -47.0, -49.0, -60.0])
def test_barrier_floor(M, orc, inp, log2_term):
    """Reading R28: a barrier term below 2^-48 counts as 0 on the GPU.  With
    every other cost weight and the noise at zero, a sample's cost is the
    barrier sum alone: one sphere is placed so that the hovering states see
    exp(-beta s) = 2^log2_term.  Above the floor the GPU matches the FP64
    oracle; below it the GPU's cost is exactly 0 while the oracle's is the
    (N+1) c_bar 2^log2_term the floor drops."""
    import math
    N = 10
    prob = inp.plain_hover(K=64, N=N, c_p=0.0, c_q=0.0, c_v=0.0, c_w=0.0, R=(0.0,) * 4, Rd=(0.0,) * 4,
                           sigma=(0.0,) * 4)
    p = prob["params"]
    beta, reach = p["beta"], 0.5 + p["r_uav"]
    s_gap = -log2_term / (beta * math.log2(math.e))  # exp(-beta s) = 2^log2_term
    d = math.sqrt(reach * reach + s_gap)
    x0 = prob["x_hat"][0:3].astype(np.float64)
    prob["obstacles"] = np.array([[x0[0] + d, x0[1], x0[2], 0.5]], np.float32)
    g = gpu_solve(M, prob)
    o = orc.mppi_step(prob, n_threads=8)
    expect = (N + 1) * p["c_bar"] * 2.0 ** log2_term
    assert np.allclose(o["costs"], expect, rtol=1e-4)  # the placement is what it says
    if log2_term >= -48.0:
        assert np.allclose(g["costs"], o["costs"], rtol=1e-4)
    else:
        assert np.all(g["costs"] == 0.0)
        assert np.all(o["costs"] > 0.0) and np.all(o["costs"] <= (N + 1) * p["c_bar"] * 2.0 ** -48)
