"""Pins of the oracle's vehicle model (Sec. III-B): Eq. drone_dynamics, the
RK4 step, the allocation matrix and the low-level constraint pipeline.

Each test checks the oracle against something other than itself: a closed
form (hover, free fall, constant spin), a conserved quantity of rigid-body
motion, a library integrator/inverse, or the matrix printed in the paper.
"""
import math

import numpy as np
import pytest


def _axis_angle(axis, theta):
    axis = np.asarray(axis, float)
    axis = axis / np.linalg.norm(axis)
    return np.concatenate([[math.cos(theta / 2)], math.sin(theta / 2) * axis])


def _hamilton(a, b):
    # Used only to build expected closed forms; the quaternion product
    # itself is pinned by test_quat_mul_matches_rotation_composition.
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _rodrigues(axis, theta):
    k = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(theta) * K + (1 - math.cos(theta)) * K @ K


def test_rotation_matrix_matches_rodrigues(orc):
    rng = np.random.default_rng(1)
    for _ in range(20):
        axis, th = rng.normal(size=3), rng.uniform(-math.pi, math.pi)
        assert np.allclose(orc.rotation_matrix(_axis_angle(axis, th)), _rodrigues(axis, th), atol=1e-13)


def test_quat_mul_matches_rotation_composition(orc):
    rng = np.random.default_rng(2)
    for _ in range(20):
        a1, t1, a2, t2 = rng.normal(size=3), rng.uniform(-3, 3), rng.normal(size=3), rng.uniform(-3, 3)
        q = orc.quat_mul(_axis_angle(a1, t1), _axis_angle(a2, t2))
        assert np.allclose(orc.rotation_matrix(q), _rodrigues(a1, t1) @ _rodrigues(a2, t2), atol=1e-13)


def test_hover_is_an_equilibrium(orc, inp):
    m = inp.model()
    x = inp.state(p=(1.0, -2.0, 3.0)).astype(float)
    xdot = orc.dynamics(m, x, m["mass"] * m["g"], [0, 0, 0])
    assert np.allclose(xdot, 0.0, atol=1e-15)
    # Through the constraint pipeline and 50 RK4 steps the state stays put.
    F, tau, wc = orc.feasible_input(m, x, [m["mass"] * m["g"], 0, 0, 0], 0.02)
    assert math.isclose(F, m["mass"] * m["g"], rel_tol=1e-14)
    assert np.allclose(tau, 0, atol=1e-15) and np.allclose(wc, 0, atol=1e-15)
    y = x.copy()
    for _ in range(50):
        y = orc.rk4_step(m, y, F, tau, 0.02)
    assert np.allclose(y, x, atol=1e-12)


def test_free_fall_is_exact_parabola(orc, inp):
    m = inp.model(motor_clip=0)
    q0 = _axis_angle([0.3, -1.0, 0.2], 0.7)
    x = np.concatenate([[1.0, 2.0, 3.0], q0, [1.0, -2.0, 0.5], [0, 0, 0]])
    h, n = 0.01, 100
    y = x.copy()
    for _ in range(n):
        y = orc.rk4_step(m, y, 0.0, [0, 0, 0], h)
    t = h * n
    g = np.array([0, 0, -m["g"]])
    assert np.allclose(y[0:3], x[0:3] + x[7:10] * t + 0.5 * g * t * t, atol=1e-12)
    assert np.allclose(y[7:10], x[7:10] + g * t, atol=1e-12)
    assert np.allclose(y[3:7], q0, atol=1e-14)


@pytest.mark.parametrize("axis,theta,expect", [
    ((1, 0, 0), math.pi / 2, (0, -1, 0)),   # roll +90 deg tips thrust to -y
    ((0, 1, 0), math.pi / 2, (1, 0, 0)),    # pitch +90 deg tips thrust to +x
    ((0, 0, 1), 1.234, (0, 0, 1)),          # yaw leaves thrust vertical
])
def test_thrust_direction_follows_attitude(orc, inp, axis, theta, expect):
    m = inp.model()
    x = np.concatenate([[0, 0, 0], _axis_angle(axis, theta), [0, 0, 0], [0, 0, 0]])
    F = 7.0
    acc = orc.dynamics(m, x, F, [0, 0, 0])[7:10]
    assert np.allclose(acc, F / m["mass"] * np.array(expect) + np.array([0, 0, -m["g"]]), atol=1e-12)


def test_constant_rate_attitude_closed_form_and_fourth_order(orc, inp):
    # Isotropic inertia: omega x J omega = 0, so omega stays constant and
    # q(t) = q0 (.) exp(omega t / 2) (body rates, right multiplication).
    m = inp.model(J=(0.01, 0.01, 0.01))
    w = np.array([1.0, 2.0, -3.0])
    q0 = _axis_angle([1, 1, 0], 0.4)
    x = np.concatenate([[0, 0, 0], q0, [0, 0, 0], w])
    T = 1.0

    def err(h):
        y = x.copy()
        for _ in range(int(round(T / h))):
            y = orc.rk4_step(m, y, m["mass"] * m["g"], [0, 0, 0], h)
        q_exact = _hamilton(q0, _axis_angle(w, np.linalg.norm(w) * T))
        assert np.allclose(y[10:13], w, atol=1e-13)
        return np.linalg.norm(y[3:7] - q_exact)

    e1, e2 = err(0.04), err(0.02)
    assert e2 < 1e-6
    assert 10.0 < e1 / e2 < 24.0  # fourth-order convergence (ratio 16)


def test_torque_free_body_conserves_world_angular_momentum(orc, inp):
    # Pins the sign of omega x J omega together with the quaternion
    # kinematics convention: L_world = R(q) J omega is constant.
    m = inp.model(J=(0.01, 0.02, 0.03))
    J = np.array(m["J"])
    w0 = np.array([1.0, 0.5, -2.0])
    x = np.concatenate([[0, 0, 0], _axis_angle([0.2, 0.1, 1], 0.3), [0, 0, 0], w0])
    L0 = orc.rotation_matrix(x[3:7]) @ (J * w0)
    E0 = 0.5 * np.dot(w0, J * w0)
    y = x.copy()
    for _ in range(2000):
        y = orc.rk4_step(m, y, m["mass"] * m["g"], [0, 0, 0], 1e-3)
    L = orc.rotation_matrix(y[3:7]) @ (J * y[10:13])
    assert np.linalg.norm(L - L0) < 1e-9 * np.linalg.norm(L0)
    assert abs(0.5 * np.dot(y[10:13], J * y[10:13]) - E0) < 1e-9 * E0
    assert not np.allclose(y[10:13], w0, atol=1e-2)  # the motion is not trivial


def test_unit_quaternion_norm_is_kept(orc, inp):
    # ||q|| = 1 (Sec. III-B) after every step, even with fast rotation.
    m = inp.model(J=(0.01, 0.02, 0.03))
    y = np.concatenate([[0, 0, 0], _axis_angle([1, 2, 3], 1.0), [0, 0, 0], [9.0, -8.0, 7.0]])
    for _ in range(200):
        y = orc.rk4_step(m, y, 10.0, [0.01, 0.0, -0.01], 0.02)
        assert abs(np.linalg.norm(y[3:7]) - 1.0) < 1e-15


def test_applied_torque_gives_euler_rate(orc, inp):
    m = inp.model()
    x = inp.state().astype(float)
    tau = np.array([0.01, -0.02, 0.003])
    assert np.allclose(orc.dynamics(m, x, 5.0, tau)[10:13], tau / np.array(m["J"]), rtol=1e-14)


def test_rk4_local_error_is_fifth_order_against_library_integrator(orc, inp):
    integrate = pytest.importorskip("scipy.integrate")
    m = inp.model(J=(0.011, 0.017, 0.029))
    x0 = np.concatenate([[0.1, -0.2, 0.3], _axis_angle([1, -2, 0.5], 0.9), [2.0, -1.0, 0.5], [1.5, -0.7, 2.2]])
    F, tau = 14.0, np.array([0.003, -0.002, 0.001])

    def ref_step(h):
        sol = integrate.solve_ivp(lambda t, y: orc.dynamics(m, y, F, tau), (0, h), x0, method="DOP853",
                                  rtol=1e-13, atol=1e-15)
        y = sol.y[:, -1]
        y[3:7] /= np.linalg.norm(y[3:7])
        return y

    e = [np.linalg.norm(orc.rk4_step(m, x0, F, tau, h) - ref_step(h)) for h in (0.04, 0.02)]
    assert e[1] < 1e-7
    assert 20.0 < e[0] / e[1] < 48.0  # local error O(h^5): ratio 32


def test_allocation_matrix_is_the_papers(orc, inp):
    m = inp.model()
    a = m["arm_l"] / math.sqrt(2)
    c = m["c_tf"]
    # Gamma as printed in Sec. III-B (X configuration).
    paper = np.array([[1, 1, 1, 1], [-a, a, a, -a], [-a, a, -a, a], [-c, -c, c, c]])
    assert np.array_equal(orc.allocation_matrix(m), paper)


def test_invert4_matches_library_inverse(orc, inp):
    rng = np.random.default_rng(3)
    G = orc.allocation_matrix(inp.model())
    assert np.allclose(orc.invert4(G), np.linalg.inv(G), rtol=1e-12, atol=1e-12)
    for _ in range(20):
        A = rng.normal(size=(4, 4))
        assert np.allclose(orc.invert4(A), np.linalg.inv(A), rtol=1e-9, atol=1e-9)


def test_feasible_input_unclipped_reproduces_desired(orc, inp):
    # No active clip: F_clip = F_t and omega_clip = omega_d (algebra of the
    # pipeline: Gamma Gamma^-1 = I and the torque is inverted exactly).
    rng = np.random.default_rng(4)
    for clip in (0, 1):
        m = inp.model(motor_clip=clip)
        for _ in range(30):
            x = np.concatenate([[0, 0, 0], _axis_angle(rng.normal(size=3), 0.5), [0, 0, 0],
                                rng.uniform(-1, 1, 3)])
            u = np.concatenate([[rng.uniform(12, 28)], x[10:13] + rng.uniform(-0.05, 0.05, 3)])
            F, tau, wc = orc.feasible_input(m, x, u, 0.01)
            assert math.isclose(F, u[0], rel_tol=1e-12)
            assert np.allclose(wc, u[1:], atol=1e-10)
            J = np.array(m["J"])
            Jw = J * x[10:13]
            tau_d = J * (u[1:] - x[10:13]) / 0.01 + np.cross(x[10:13], Jw)
            assert np.allclose(tau, tau_d, rtol=1e-10, atol=1e-12)


def test_feasible_input_clipped_respects_rotor_limits(orc, inp):
    m = inp.model(motor_clip=1)
    G = np.array(orc.allocation_matrix(m))
    x = inp.state().astype(float)
    # A large roll-rate demand saturates the rotors.
    F, tau, wc = orc.feasible_input(m, x, [20.0, 9.0, 0.0, 0.0], 0.01)
    T = np.linalg.solve(G, np.concatenate([[F], tau]))
    assert np.all(T >= m["T_min"] - 1e-9) and np.all(T <= m["T_max"] + 1e-9)
    assert np.any(np.isclose(T, m["T_min"])) or np.any(np.isclose(T, m["T_max"]))
    assert 0 < wc[0] < 9.0  # moves toward the demand but cannot reach it in one step
    assert 4 * m["T_min"] - 1e-9 <= F <= 4 * m["T_max"] + 1e-9
    # Whole thrust range beyond the rotors' limits is cut to the box of 4 rotors.
    F2, _, _ = orc.feasible_input(m, x, [100.0, 0, 0, 0], 0.01)
    assert math.isclose(F2, 4 * m["T_max"], rel_tol=1e-12)
    F3, _, _ = orc.feasible_input(m, x, [0.0, 0, 0, 0], 0.01)
    assert math.isclose(F3, 4 * m["T_min"], rel_tol=1e-12)


def test_clamp_input_box(orc, inp):
    m = inp.model()
    assert np.allclose(orc.clamp_input(m, [50.0, 11.0, -12.0, 3.0]), [m["F_max"], 10.0, -10.0, 3.0])
    assert np.allclose(orc.clamp_input(m, [-1.0, 0.0, 0.0, -10.5]), [m["F_min"], 0.0, 0.0, -10.0])


def test_quaternion_distance_properties(orc):
    rng = np.random.default_rng(5)
    for _ in range(20):
        q = _axis_angle(rng.normal(size=3), rng.uniform(-3, 3))
        for metric in (0, 1):
            assert abs(orc.quat_distance(q, q, metric)) < 1e-7
            assert abs(orc.quat_distance(q, -q, metric)) < 1e-7
        th = rng.uniform(0, math.pi)
        q2 = _hamilton(q, _axis_angle(rng.normal(size=3), th))
        assert math.isclose(orc.quat_distance(q, q2, 0), math.sin(th / 2) ** 2, rel_tol=1e-10, abs_tol=1e-12)
        assert math.isclose(orc.quat_distance(q, q2, 1), th, rel_tol=1e-6, abs_tol=1e-6)
    # 360 degree single-axis sweep: peak at 180 degrees, back to 0 at 360.
    ang = np.linspace(0, 2 * math.pi, 361)
    d0 = [orc.quat_distance([1, 0, 0, 0], _axis_angle([0, 0, 1], a), 0) for a in ang]
    d1 = [orc.quat_distance([1, 0, 0, 0], _axis_angle([0, 0, 1], a), 1) for a in ang]
    assert int(np.argmax(d0)) == 180 and int(np.argmax(d1)) == 180
    assert math.isclose(d0[180], 1.0) and math.isclose(d1[180], math.pi, rel_tol=1e-6)
    assert abs(d0[-1]) < 1e-12 and abs(d1[-1]) < 1e-6


def test_rho_ref_weights_each_block(orc, inp):
    p = inp.params(c_p=3.0, c_q=5.0, c_v=7.0, c_w=11.0)
    ref = np.concatenate([[1, 2, 3], _axis_angle([0, 0, 1], 0.3), [0.1, 0.2, 0.3], [0.4, 0.5, 0.6]])
    x = ref.copy()
    assert abs(orc.rho_ref(p, x, ref)) < 1e-12
    x = ref.copy(); x[0:3] += [1, 2, 2]
    assert math.isclose(orc.rho_ref(p, x, ref), 3.0 * 9)
    x = ref.copy(); x[7:10] += [0, 3, 4]
    assert math.isclose(orc.rho_ref(p, x, ref), 7.0 * 25)
    x = ref.copy(); x[10:13] += [1, 0, 0]
    assert math.isclose(orc.rho_ref(p, x, ref), 11.0)
    x = ref.copy(); x[3:7] = _hamilton(ref[3:7], _axis_angle([1, 0, 0], math.pi / 2))
    assert math.isclose(orc.rho_ref(p, x, ref), 5.0 * 0.5 ** 2, rel_tol=1e-12)
