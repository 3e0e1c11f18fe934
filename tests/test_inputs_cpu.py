"""The seeded synthetic workloads have the shapes and value ranges their
recipes state (the stand-ins for the paper's simulator trajectories and
obstacle maps), and are reproducible from their seeds."""
import math

import numpy as np


def _obstacles_in(obs, lo, hi, rmin, rmax):
    c, r = obs[:, :3], np.abs(obs[:, 3])
    return bool(np.all(c >= np.array(lo) - 1e-5) and np.all(c <= np.array(hi) + 1e-5) and np.all(r >= rmin - 1e-6)
                and np.all(r <= rmax + 1e-6))


def test_problem_layout_and_f32(inp):
    p = inp.eight_with_spheres(K=512, N=20, M=7)
    assert p["x_hat"].shape == (13,) and p["ref"].shape == (21, 13) and p["u_nom"].shape == (20, 4)
    assert p["obstacles"].shape == (7, 4)
    for k in ("x_hat", "ref", "obstacles", "u_nom"):
        assert p[k].dtype == np.float32 and p[k].flags.c_contiguous
    # Every floating parameter is exactly representable in FP32 (both sides
    # of the parity tests see the same numbers).
    for d in (p["model"], p["params"]):
        for v in d.values():
            for x in (v if isinstance(v, tuple) else (v,)):
                if isinstance(x, float):
                    assert float(np.float32(x)) == x
    # Reference attitudes are unit quaternions; the start is the reference.
    assert np.allclose(np.linalg.norm(p["ref"][:, 3:7], axis=1), 1.0, atol=1e-6)
    assert np.array_equal(p["x_hat"], p["ref"][0])


def test_headline_recipe(inp):
    p = inp.eight_with_spheres()
    assert (p["params"]["K"], p["params"]["N"]) == (16384, 100) and p["params"]["dt"] == np.float32(0.01)
    assert p["model"]["motor_clip"] == 1
    assert _obstacles_in(p["obstacles"], (-20, -10, 0), (20, 10, 5), 0.3, 1.0)
    assert np.all(p["obstacles"][:, 3] > 0)  # spheres only
    # Hover nominal: collective thrust m g, zero body rates.
    assert np.allclose(p["u_nom"][:, 0], p["model"]["mass"] * p["model"]["g"], rtol=1e-6)
    assert np.all(p["u_nom"][:, 1:] == 0)


def test_stress_recipe(inp):
    p = inp.stress_line(K=1024, N=50)
    o = p["obstacles"]
    assert o.shape == (1024, 4)
    assert np.sum(o[:, 3] > 0) == 512 and np.sum(o[:, 3] < 0) == 512  # spheres, vertical cylinders
    assert _obstacles_in(o, (0, 0, 0), (100, 100, 10), 0.2, 1.5)


def test_batched_recipe_ranges_and_reproducibility(inp):
    probs = inp.batched_uneven(n=256)
    K = np.array([q["params"]["K"] for q in probs])
    N = np.array([q["params"]["N"] for q in probs])
    M = np.array([q["obstacles"].shape[0] for q in probs])
    assert K.min() >= 1024 and K.max() <= 32768
    assert N.min() >= 30 and N.max() <= 150 and M.min() >= 0 and M.max() <= 128
    # log-uniform K: log2 K roughly uniform on [10, 15]
    lk = np.log2(K)
    assert abs(lk.mean() - 12.5) < 0.3 and np.sum(lk < 12.5) / len(lk) > 0.35
    # Distinct noise streams per vehicle, and the same draw from the same seed.
    keys = {(q["params"]["seed"], q["params"]["stream_id"]) for q in probs}
    assert len(keys) == len(probs)
    again = inp.batched_uneven(n=256)
    assert all(np.array_equal(a["x_hat"], b["x_hat"]) and np.array_equal(a["obstacles"], b["obstacles"])
               and a["params"] == b["params"] for a, b in zip(probs, again))
    # Start states are perturbed around the reference: at most 1 m away.
    for q in probs[:32]:
        assert np.all(np.abs(q["x_hat"][0:3] - q["ref"][0, 0:3]) <= 1.0 + 1e-5)


def test_serving_fleet_recipe(inp):
    fleet = inp.serving_fleet(n_vehicles=300)
    assert {v["K"] for v in fleet} <= {2048, 8192, 32768} and {v["N"] for v in fleet} <= {50, 100}
    assert all(v["obstacles"].shape == (32, 4) for v in fleet)
    assert len({v["stream_id"] for v in fleet}) == 300
    # Each choice appears (uniform draws over 300 vehicles).
    assert {v["K"] for v in fleet} == {2048, 8192, 32768} and {v["N"] for v in fleet} == {50, 100}
    assert all(0.0 <= v["phase"] < 2 * math.pi for v in fleet)
