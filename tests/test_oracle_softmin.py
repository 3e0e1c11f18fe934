"""Pins of the oracle's weighting, update, apply and shift (Sec. III-A
Eq. cost_2, Eq. u_update, Alg. 1; Sec. IV-B interpolation; Sec. IV-E delay
compensation) against the limits the paper states and closed forms.
"""
import math

import numpy as np
import pytest


def test_weights_normalised_nonnegative_and_shift_invariant(orc):
    rng = np.random.default_rng(0)
    S = rng.uniform(100.0, 130.0, 257)
    rc, w = orc.weights(S, 3.0)
    assert rc == 0 and np.all(w >= 0) and math.isclose(w.sum(), 1.0, rel_tol=1e-14)
    # Subtracting rho "does not change the result" (Sec. III-A): any shift.
    for c in (-99.0, 1e3, 12345.678):
        assert np.allclose(orc.weights(S + c, 3.0)[1], w, rtol=1e-9, atol=1e-300)
    # Scaling costs and temperature together leaves weights unchanged.
    assert np.allclose(orc.weights(S * 4.0, 12.0)[1], w, rtol=1e-9, atol=1e-300)


def test_two_sample_closed_form(orc):
    for S1, S2, lam in [(1.0, 2.0, 1.0), (5.0, 3.5, 0.7), (10.0, 10.0, 2.0)]:
        w = orc.weights([S1, S2], lam)[1]
        assert math.isclose(w[0], 1.0 / (1.0 + math.exp(-(S2 - S1) / lam)), rel_tol=1e-14)


def test_temperature_limits(orc):
    rng = np.random.default_rng(1)
    S = rng.uniform(0.0, 50.0, 100)
    w0 = orc.weights(S, 1e-30)[1]
    assert w0[np.argmin(S)] == 1.0 and np.count_nonzero(w0) == 1  # best rollout only
    winf = orc.weights(S, 1e30)[1]
    assert np.allclose(winf, 1.0 / S.size, rtol=1e-12)  # plain average
    tie = orc.weights([2.0, 1.0, 1.0, 5.0], 1e-30)[1]
    assert np.allclose(tie, [0.0, 0.5, 0.5, 0.0])  # ties share equally


def test_nonfinite_costs(orc):
    rc, w = orc.weights([np.nan, 3.0, np.inf, 4.0], 1.0)
    assert rc == 0 and w[0] == 0.0 and w[2] == 0.0 and math.isclose(w[1] + w[3], 1.0)
    rc, _ = orc.weights([np.nan, np.inf], 1.0)
    assert rc == orc.ENONFINITE


@pytest.fixture
def small(inp):
    m = inp.model(motor_clip=1)
    p = inp.params(K=40, N=6, dt=0.02, seed=11, stream_id=1, **{"lambda": 50.0})
    ref = inp.Trajectory("eight").window(0.3, p["N"], p["dt"])
    x = ref[0].copy()
    x[0] += 0.4
    obs = np.array([[x[0] + 1.0, x[1], x[2], 0.4]], np.float32)
    return inp.problem(m, p, x, ref, obs, inp.hover_u(m, p["N"]), it=9)


def _deltas(orc, prob):
    p = prob["params"]
    return orc.noise_block(p, prob["iter"], p["K"], p["N"])


def test_costs_are_the_rollouts_and_update_is_weighted_noise(orc, small):
    out = orc.mppi_step(small)
    K = small["params"]["K"]
    S = np.array([orc.rollout(small, k) for k in range(K)])
    assert np.array_equal(out["costs"], S)
    rc, w = orc.weights(S, small["params"]["lambda"])
    assert np.allclose(out["weights"], w, rtol=0, atol=0)
    expect = small["u_nom"].astype(float) + np.einsum("k,kjc->jc", w, _deltas(orc, small))
    assert np.allclose(out["u_out"], expect, rtol=1e-13, atol=1e-13)
    assert 1.5 < 1.0 / np.sum(w ** 2) < K  # several samples contribute


def test_single_sample_returns_its_controls(orc, small):
    prob = dict(small, params=dict(small["params"], K=1))
    out = orc.mppi_step(prob)
    assert np.allclose(out["u_out"], small["u_nom"] + _deltas(orc, prob)[0], rtol=0, atol=1e-15)


def test_lambda_to_zero_returns_best_sample(orc, small):
    prob = dict(small, params=dict(small["params"], **{"lambda": 1e-30}))
    out = orc.mppi_step(prob)
    best = int(np.argmin(out["costs"]))
    assert np.allclose(out["u_out"], small["u_nom"] + _deltas(orc, prob)[best], rtol=0, atol=1e-15)


def test_lambda_to_infinity_returns_mean_perturbation(orc, small):
    prob = dict(small, params=dict(small["params"], **{"lambda": 1e30}))
    out = orc.mppi_step(prob)
    assert np.allclose(out["u_out"], small["u_nom"] + _deltas(orc, prob).mean(axis=0), rtol=1e-12, atol=1e-13)


def test_zero_noise_returns_nominal(orc, small):
    prob = dict(small, params=dict(small["params"], sigma=(0.0, 0.0, 0.0, 0.0)))
    out = orc.mppi_step(prob)
    assert np.array_equal(out["u_out"], small["u_nom"].astype(float))
    assert np.all(out["costs"] == out["costs"][0])
    assert np.allclose(out["weights"], 1.0 / prob["params"]["K"])


def test_shift_tail_and_interpolation(orc, small, inp):
    out = orc.mppi_step(small)
    m = small["model"]
    u = out["u_out"]
    hover = np.array([m["mass"] * m["g"], 0, 0, 0])
    assert np.array_equal(out["u_next"], np.vstack([u[1:], hover]))
    rep = orc.mppi_step(dict(small, params=dict(small["params"], tail_mode=1)))
    assert np.array_equal(rep["u_next"], np.vstack([u[1:], u[-1:]]))
    half = orc.mppi_step(dict(small, params=dict(small["params"], shift_alpha=0.25)))
    later = np.vstack([u[1:], hover])
    assert np.allclose(half["u_next"], 0.75 * u + 0.25 * later, rtol=1e-15, atol=1e-15)


def test_apply_command_is_feasible_input_of_first_control(orc, small):
    out = orc.mppi_step(small)
    m, p = small["model"], small["params"]
    u0 = orc.clamp_input(m, out["u_out"][0])
    F, tau, wc = orc.feasible_input(m, small["x_hat"], u0, p["dt"])
    assert np.allclose(out["u_cmd"], np.concatenate([[F], wc]), rtol=0, atol=0)
    assert np.allclose(out["x_next"], orc.rk4_step(m, small["x_hat"], F, tau, p["dt"]), rtol=0, atol=0)


def test_nonfinite_state_keeps_nominal(orc, small):
    x = small["x_hat"].copy()
    x[7] = np.nan
    out = orc.mppi_step(dict(small, x_hat=x))
    assert out["status"] == orc.ENONFINITE
    assert np.array_equal(out["u_out"], small["u_nom"].astype(float))


def test_delay_compensation_starts_rollouts_from_prediction(orc, small):
    delay = 0.004
    prob = dict(small, params=dict(small["params"], delay=delay))
    out = orc.mppi_step(prob)
    m, p = small["model"], small["params"]
    F, tau, _ = orc.feasible_input(m, small["x_hat"], orc.clamp_input(m, small["u_nom"][0]), p["dt"])
    x_pred = orc.rk4_step(m, small["x_hat"], F, tau, delay)
    for k in (0, 17, 39):
        assert out["costs"][k] == orc.rollout(small, k, x0=x_pred)
