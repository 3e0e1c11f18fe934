"""Pins of the oracle's rollout cost (Sec. IV-C Eq. cost / rho_ref,
Sec. IV-D obstacle term) on rollouts whose trajectory has a closed form.

With sigma = 0 every rollout follows the nominal controls exactly, so a
hover or a piecewise-constant vertical thrust sequence gives a trajectory
known from kinematics (RK4 is exact for piecewise-constant acceleration),
and the cost sum is written out from that trajectory.  These pin the index
ranges of the sums (j = 0..N for state terms, 0..N-1 for the input term,
0..N-2 for the rate term), which reference sample pairs with which state,
and the obstacle geometry.
"""
import math

import numpy as np
import pytest


def _quiet(inp, K=1, N=12, dt=0.05, clip=0, **over):
    m = inp.model(motor_clip=clip)
    p = inp.params(K=K, N=N, dt=dt, sigma=(0.0, 0.0, 0.0, 0.0), **over)
    return m, p


def test_hover_offset_cost_closed_form(orc, inp):
    for clip in (0, 1):
        m, p = _quiet(inp, clip=clip)
        N = p["N"]
        x0 = inp.state(p=(0.5, -0.25, 0.125))
        ref = inp.Trajectory("hover").window(0.0, N, p["dt"])
        u = inp.hover_u(m, N)
        prob = inp.problem(m, p, x0, ref, np.zeros((0, 4)), u)
        S = orc.rollout(prob, 0)
        d2 = 0.5 ** 2 + 0.25 ** 2 + 0.125 ** 2
        uh = float(u[0, 0])
        expect = (N + 1) * p["c_p"] * d2 + N * p["R"][0] * uh * uh
        assert math.isclose(S, expect, rel_tol=1e-12)


def test_moving_reference_pairs_state_j_with_reference_j(orc, inp):
    m, p = _quiet(inp, N=9)
    N, dt = p["N"], p["dt"]
    c = 2.0
    ref = np.zeros((N + 1, 13), np.float32)
    ref[:, 3] = 1.0
    ref[:, 0] = c * dt * np.arange(N + 1)  # reference slides along +x (v_ref = 0 on purpose)
    u = inp.hover_u(m, N)
    prob = inp.problem(m, p, inp.state(), ref, np.zeros((0, 4)), u)
    S = orc.rollout(prob, 0)
    expect = sum(p["c_p"] * float(ref[j, 0]) ** 2 for j in range(N + 1)) + N * p["R"][0] * float(u[0, 0]) ** 2
    assert math.isclose(S, expect, rel_tol=1e-12)


def test_vertical_thrust_sequence_cost_closed_form(orc, inp):
    m, p = _quiet(inp, N=10, dt=0.05)
    N, dt, g = p["N"], p["dt"], m["g"]
    acc = np.array([(1.5 if j % 3 == 0 else -0.75) for j in range(N)])
    u = np.zeros((N, 4), np.float32)
    u[:, 0] = (m["mass"] * (g + acc)).astype(np.float32)
    a_eff = u[:, 0].astype(float) / m["mass"] - g
    ref = inp.Trajectory("hover").window(0.0, N, dt)
    prob = inp.problem(m, p, inp.state(), ref, np.zeros((0, 4)), u)
    S, traj, useq, _ = orc.rollout(prob, 0, want_traj=True)
    # Kinematics with piecewise-constant acceleration.
    z, v = [0.0], [0.0]
    for j in range(N):
        z.append(z[-1] + v[-1] * dt + 0.5 * a_eff[j] * dt * dt)
        v.append(v[-1] + a_eff[j] * dt)
    assert np.allclose(traj[:, 2], z, atol=1e-12) and np.allclose(traj[:, 9], v, atol=1e-12)
    F = u[:, 0].astype(float)
    expect = sum(p["c_p"] * z[j] ** 2 + p["c_v"] * v[j] ** 2 for j in range(N + 1))
    expect += sum(p["R"][0] * F[j] ** 2 for j in range(N))
    expect += sum(p["Rd"][0] * (F[j + 1] - F[j]) ** 2 for j in range(N - 1))
    assert math.isclose(S, expect, rel_tol=1e-11)


def test_attitude_term_in_rollout(orc, inp):
    m, p = _quiet(inp, N=6)
    N = p["N"]
    ref = inp.Trajectory("hover").window(0.0, N, p["dt"])
    ref[:, 3:7] = [math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]  # 90 deg yaw
    u = inp.hover_u(m, N)
    prob = inp.problem(m, p, inp.state(), ref, np.zeros((0, 4)), u)
    d = math.sin(math.pi / 4) ** 2  # 1 - <q, q_ref>^2 = sin^2(45 deg)
    expect = (N + 1) * p["c_q"] * d * d + N * p["R"][0] * float(u[0, 0]) ** 2
    assert math.isclose(orc.rollout(prob, 0), expect, rel_tol=1e-6)


@pytest.mark.parametrize("inside", [False, True])
def test_sphere_and_cylinder_cost(orc, inp, inside):
    m, p = _quiet(inp, N=5)
    N = p["N"]
    ref = inp.Trajectory("hover").window(0.0, N, p["dt"])
    u = inp.hover_u(m, N)
    base = inp.problem(m, p, inp.state(), ref, np.zeros((0, 4)), u)
    S0 = orc.rollout(base, 0)
    d, r = (0.9, 1.0) if inside else (2.0, 0.5)
    gap = d * d - (r + p["r_uav"]) ** 2
    per_state = p["c_bar"] * math.exp(-p["beta"] * max(gap, 0.0)) + (p["c_obs"] if gap <= 0 else 0.0)
    sph = inp.problem(m, p, inp.state(), ref, np.array([[d, 0.0, 0.0, r]]), u)
    assert math.isclose(orc.rollout(sph, 0) - S0, (N + 1) * per_state, rel_tol=1e-9)
    # A vertical pillar ignores the height of its centre.
    cyl = inp.problem(m, p, inp.state(), ref, np.array([[0.0, d, 123.0, -r]]), u)
    assert math.isclose(orc.rollout(cyl, 0) - S0, (N + 1) * per_state, rel_tol=1e-9)
    # The same offset in z does count for a sphere.
    far = inp.problem(m, p, inp.state(), ref, np.array([[0.0, 0.0, 10.0, r]]), u)
    assert orc.rollout(far, 0) - S0 < 1e-6


def test_collision_indicator_counts_once_per_state(orc, inp):
    m, p = _quiet(inp, N=4)
    N = p["N"]
    ref = inp.Trajectory("hover").window(0.0, N, p["dt"])
    u = inp.hover_u(m, N)
    base = orc.rollout(inp.problem(m, p, inp.state(), ref, np.zeros((0, 4)), u), 0)
    two = np.array([[0.1, 0.0, 0.0, 1.0], [-0.1, 0.0, 0.0, -1.0]])
    S = orc.rollout(inp.problem(m, p, inp.state(), ref, two, u), 0)
    assert math.isclose(S - base, (N + 1) * (2 * p["c_bar"] + p["c_obs"]), rel_tol=1e-12)


def test_rollout_of_noise_uses_sample_noise_and_clamp(orc, inp):
    # The controls of sample k are clamp(u_nom_j + delta_j^k) and the
    # rollout with them equals the rollout of a zero-noise problem whose
    # nominal is exactly those controls.
    m = inp.model(motor_clip=1)
    p = inp.params(K=8, N=7, dt=0.02, sigma=(8.0, 6.0, 6.0, 6.0), seed=3)
    N = p["N"]
    ref = inp.Trajectory("eight").window(0.0, N, p["dt"])
    u = inp.hover_u(m, N)
    prob = inp.problem(m, p, ref[0], ref, np.zeros((0, 4)), u, it=5)
    S, traj, useq, _ = orc.rollout(prob, 6, want_traj=True)
    for j in range(N):
        d = orc.noise(p, 5, 6, j)
        assert np.allclose(useq[j], orc.clamp_input(m, u[j] + d), atol=0)
    assert np.any(useq[:, 1:] == 10.0) or np.any(useq[:, 1:] == -10.0)  # clamp active somewhere
    quiet = dict(p, sigma=(0.0, 0.0, 0.0, 0.0))
    replay = dict(prob, params=quiet, u_nom=useq)  # float64 controls, no rounding
    S2, traj2, _, _ = orc.rollout(replay, 0, want_traj=True)
    assert np.allclose(traj, traj2, atol=1e-12) and math.isclose(S, S2, rel_tol=1e-12)


def _grid_params(p):
    occ = np.zeros((4, 5, 6), np.uint8)  # (z, y, x), voxel 0.5 m, origin (-1, -1, -1)
    occ[2, 2, 3] = 1  # covers x in [0.5, 1), y in [0, 0.5), z in [0, 0.5)
    return dict(p, grid={"occ": occ, "origin": (-1.0, -1.0, -1.0), "voxel": 0.5})


def test_grid_occupancy_lookup(orc, inp):
    p = _grid_params(inp.params())
    assert orc.grid_occupied(p, (0.75, 0.25, 0.25))[0] == 1
    assert orc.grid_occupied(p, (0.5, 0.0, 0.0))[0] == 1  # lower faces belong to the voxel
    assert orc.grid_occupied(p, (1.0, 0.25, 0.25))[0] == 0  # upper face belongs to the next one
    assert orc.grid_occupied(p, (0.25, 0.25, 0.25))[0] == 0
    assert orc.grid_occupied(p, (0.25, 0.75, 0.25))[0] == 0  # swapped x/y would hit here
    assert orc.grid_occupied(p, (0.25, 0.25, 0.75))[0] == 0  # swapped x/z would hit here
    assert orc.grid_occupied(p, (5.0, 0.25, 0.25))[0] == 0  # outside the grid: free
    assert orc.grid_occupied(p, (-1.25, 0.25, 0.25))[0] == 0
    occ, face = orc.grid_occupied(p, (0.75, 0.3, 0.1))
    assert occ == 1 and abs(face - 0.1) < 1e-12  # nearest occupancy-changing face is z = 0
    occ, face = orc.grid_occupied(p, (-0.6, -0.6, -0.6))
    assert occ == 0 and face == float("inf")  # neighbours all free


@pytest.mark.parametrize("inside", [False, True])
def test_grid_indicator_in_rollout_once_per_state(orc, inp, inside):
    m, p = _quiet(inp, N=5)
    N = p["N"]
    p = _grid_params(p)
    x = inp.state(p=(0.75, 0.25, 0.25) if inside else (0.25, 0.25, 0.25))
    ref = inp.Trajectory("hover", {"at": tuple(x[:3])}).window(0.0, N, p["dt"])
    u = inp.hover_u(m, N)
    base = orc.rollout(inp.problem(m, dict(p, grid=None), x, ref, np.zeros((0, 4)), u), 0)
    S = orc.rollout(inp.problem(m, p, x, ref, np.zeros((0, 4)), u), 0)
    assert math.isclose(S - base, (N + 1) * p["c_obs"] if inside else 0.0, rel_tol=1e-12, abs_tol=1e-9)
    # A sphere around the same state: still one indicator per state.
    sph = np.array([[x[0], x[1], x[2], 0.3]], np.float32)
    S2 = orc.rollout(inp.problem(m, p, x, ref, sph, u), 0)
    S3 = orc.rollout(inp.problem(m, dict(p, grid=None), x, ref, sph, u), 0)
    assert math.isclose(S2, S3, rel_tol=1e-12)
