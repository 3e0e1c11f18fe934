"""Pins against values the paper prints (fixtures under tests/golden/, each
file citing its table or section).

- the allocation matrix Gamma of Sec. III-B against the oracle's;
- Table I's vehicle through the oracle's constraint pipeline: the rotor
  limits fix the collective-thrust range (4 T_min .. 4 T_max) and the yaw
  torque a saturated demand can reach, and hover must need no clipping;
- Table I and Table II against the parameter tables the synthetic
  workloads are built from;
- Table III's peak speed and acceleration against the synthetic reference
  trajectories that stand in for the paper's.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.lstrip().startswith("#")]


def _table(name):
    return {r[0]: [float(v) for v in r[1:]] for r in _rows(name)}


@pytest.fixture(scope="module")
def table1():
    return _table("table1_vehicle.txt")


@pytest.fixture(scope="module")
def table2():
    return _table("table2_mppi.txt")


def test_allocation_matrix_matches_printed_gamma(orc, inp, table1):
    m = inp.model(**inp.TABLE_I_VEHICLE)
    unit = {"1": 1.0, "l/sqrt2": table1["arm_l_m"][0] / math.sqrt(2.0), "c_tf": table1["c_tf_m"][0]}
    rows = _rows("allocation_matrix.txt")
    assert [r[0] for r in rows] == ["unit"] * 4
    gamma = np.array([[unit[r[1]] * float(v) for v in r[2:]] for r in rows])
    # The fixture's l and c_tf are the decimal values; the oracle sees the
    # model's float32-rounded ones.
    assert np.allclose(orc.allocation_matrix(m), gamma, rtol=1e-7, atol=0.0)


def test_table1_vehicle_hover_needs_no_clipping(orc, inp, table1):
    m = inp.model(**inp.TABLE_I_VEHICLE)
    mg = m["mass"] * m["g"]
    # Hover: each rotor carries m g / 4 = 2.97 N, inside [0.3, 19] N.
    assert table1["T_min_N"][0] < mg / 4 < table1["T_max_N"][0]
    F, tau, wc = orc.feasible_input(m, inp.state().astype(float), [mg, 0.0, 0.0, 0.0], 0.1)
    assert math.isclose(F, mg, rel_tol=1e-12)
    assert np.allclose(tau, 0.0, atol=1e-12) and np.allclose(wc, 0.0, atol=1e-12)


def test_table1_vehicle_thrust_range_is_four_rotors(orc, inp, table1):
    m = inp.model(**inp.TABLE_I_VEHICLE)
    x = inp.state().astype(float)
    t_min, t_max = table1["T_min_N"][0], table1["T_max_N"][0]
    F_hi, tau_hi, _ = orc.feasible_input(m, x, [500.0, 0.0, 0.0, 0.0], 0.1)
    F_lo, tau_lo, _ = orc.feasible_input(m, x, [0.0, 0.0, 0.0, 0.0], 0.1)
    assert math.isclose(F_hi, 4 * t_max, rel_tol=1e-7)  # 76 N
    assert math.isclose(F_lo, 4 * t_min, rel_tol=1e-7)  # 1.2 N
    assert np.allclose(tau_hi, 0.0, atol=1e-9) and np.allclose(tau_lo, 0.0, atol=1e-9)


def test_table1_vehicle_saturated_yaw_torque(orc, inp, table1):
    # A huge yaw-rate demand at hover thrust drives rotors 1, 2 to T_min and
    # 3, 4 to T_max (the c_tf row of Gamma is -,-,+,+), so the clipped input
    # is F = 2 (T_min + T_max), tau = (0, 0, 2 c_tf (T_max - T_min)).
    m = inp.model(**inp.TABLE_I_VEHICLE)
    t_min, t_max, c = table1["T_min_N"][0], table1["T_max_N"][0], table1["c_tf_m"][0]
    F, tau, wc = orc.feasible_input(m, inp.state().astype(float), [m["mass"] * m["g"], 0.0, 0.0, 1e4], 0.1)
    assert math.isclose(F, 2 * (t_min + t_max), rel_tol=1e-7)
    assert np.allclose(tau[:2], 0.0, atol=1e-9)
    assert math.isclose(tau[2], 2 * c * (t_max - t_min), rel_tol=1e-6)
    # omega_clip = omega + J^-1 tau_clip dt (no gyroscopic term at rest).
    assert math.isclose(wc[2], tau[2] / m["J"][2] * 0.1, rel_tol=1e-12)


def test_parameter_tables_are_the_papers(inp, table1, table2):
    v, p = inp.TABLE_I_VEHICLE, inp.PARAMS_DEFAULT
    assert v["mass"] == table1["mass_kg"][0]
    for d in (v, inp.MODEL_DEFAULT):
        assert d["arm_l"] == table1["arm_l_m"][0] and d["c_tf"] == table1["c_tf_m"][0]
        assert np.allclose(d["J"], np.array(table1["J_diag_g_m2"]) * 1e-3, rtol=1e-12)
        assert d["T_min"] == table1["T_min_N"][0]
    assert v["T_max"] == table1["T_max_N"][0]
    assert tuple(v["w_max"]) == (table1["w_xy_max_rad_s"][0],) * 2 + (table1["w_z_max_rad_s"][0],)
    for key, name in (("c_p", "c_p"), ("c_v", "c_v"), ("c_q", "c_q"), ("c_w", "c_w")):
        assert p[key] == table2[name][0]
    assert tuple(p["R"]) == tuple(table2["R"]) and tuple(p["Rd"]) == tuple(table2["R_Delta"])
    t = inp.TABLE_II_MPPI
    assert (t["dt"], t["K"], t["N"], t["lambda"]) == (table2["dt_s"][0], table2["K"][0], table2["N"][0],
                                                      table2["lambda"][0])
    assert tuple(t["Sigma"]) == tuple(table2["Sigma"])


def test_operating_point_problem_uses_table2(inp, table2):
    for t1 in (False, True):
        prob = inp.paper_operating_point(table1_vehicle=t1)
        p = prob["params"]
        assert (p["K"], p["N"]) == (int(table2["K"][0]), int(table2["N"][0]))
        assert p["dt"] == np.float32(table2["dt_s"][0]) and p["lambda"] == np.float32(table2["lambda"][0])
        # Sigma is a covariance: the generator's standard deviations square to it.
        assert np.allclose(np.square(np.float64(p["sigma"])), table2["Sigma"], rtol=1e-6)
        assert prob["ref"].shape == (16, 13) and prob["u_nom"].shape == (15, 4)
        assert prob["model"]["mass"] == np.float32(1.21 if t1 else 1.0)


def _peaks(traj, period):
    ts = np.linspace(0.0, period, 20001)
    v = max(np.linalg.norm(traj.pva(t)[1]) for t in ts)
    a = max(np.linalg.norm(traj.pva(t)[2]) for t in ts)
    return v, a


def test_synthetic_trajectories_match_table3_magnitudes(inp):
    t3 = {r[0]: (float(r[1]), float(r[2])) for r in _rows("table3_trajectories.txt")}
    # The line stands in for the paper's fastest trajectory: both peaks
    # within 3 %.
    line = inp.Trajectory("line")
    v, a = _peaks(line, 2 * math.pi / 1.6667)
    assert abs(v / t3["line"][0] - 1) < 0.03 and abs(a / t3["line"][1] - 1) < 0.03
    # The figure eight keeps the paper's peak acceleration (within 2 %) at a
    # higher peak speed (12 m/s against 8.853 m/s).
    eight = inp.Trajectory("eight")
    v, a = _peaks(eight, 2 * math.pi / 0.4243)
    assert abs(a / t3["eight"][1] - 1) < 0.02
    assert 11.9 < v < 12.1 and v > t3["eight"][0]
